// kt_stage.cuh -- the fused KT + Heun stage kernel (one launch per Runge-Kutta stage).
//
// One thread owns one physical cell and performs, in order (Sec. 4.3 steps 1-4 / 5-8):
//   a) for x, y, eta: generalised-minmod slopes of the 15 conserved components and of u^tau,
//      u^d on the 5-point stencil; half-cell extrapolations; local speeds a = max(|v+|,|v-|);
//      central-upwind fluxes at both faces; -(H_{i+1/2} - H_{i-1/2})/dx       (Eqs. Hflux, ax)
//   b) the source vector J = S + G of App. B: central differences of v P - v pi^{tau nu} +
//      pi^{d nu}, the geometric terms, and the relaxation sources built from theta, D u,
//      sigma, omega (App. A) with the coefficients of Eqs. (betaPi)-(lambdapiPi)
//   c) the Heun update in FP64: q* = q + dtau C[q]   or   q^{n+1} = (q^n + q* + dtau C[q*])/2
//   d) the FP64 inversion T^{tau mu} -> (e, u^mu) of Eq. (eInferred) at tau^{n+1}
//   e) the regulator of Eq. (regPimunu)
//   f) stores, including the ghost copies owned by boundary cells (Eqs. ghostCells_1/2)
// R is the arithmetic type of a) and b): double (KT_FP64) or float (KT_MIXED).
#pragma once
#include "kt_device.cuh"
#include "kt_mlp.cuh"

namespace kt {

template <typename R>
struct StageIO {
  const double* q_in;    // 15 fields, FP64 (q^n or q^*), read at the own cell for the Heun update
  const double* q_base;  // stage 2: q^n, read at the own cell only (aliases q_out)
  double* q_out;
  const R* qr_in;        // 15 fields in the stencil precision (FP64 mode: q_in itself; mixed: an
  R* qr_out;             // FP32 copy written by the previous stage); qr_out null in FP64 mode
  const R* u_in;         // 4 fields, stencil input (u^n or u^*)
  const R* u_prev;       // 4 fields, own cell only: u^{n-1} (stage 1) or u^n (stage 2)
  R* u_out;              // may alias u_prev (own cell only)
  const R* e_in;
  const R* p_in;
  R* e_out;
  R* p_out;
  const double* d_tau;   // tau^n
  unsigned* status;
  unsigned* max_speed_bits;
  unsigned long long* counters;  // [0] Newton iterations, [1] regulated cells, [2] fallbacks
  const uint32_t* mlp_packed;  // learned start: packed weights (see kt_mlp.cuh), or null
  float* reg_out;        // stage 2: the regulation factor applied to pi^{n+1} at each cell, or null
};

// ------------------------------------------------------------------ a) the stencil
// Per direction d the cell has two faces, L = i-1/2 and R = i+1/2, each with a left (m) and a
// right (p) state.  With F = v q the central-upwind flux of Eq. (Hflux) is linear in the face
// states, H = (v^p - a)/2 q^p + (v^m + a)/2 q^m, so the velocities and speeds of a face are
// folded once into four weights per direction (times 1/dx, the R-face weights negated),
//   -(H_R - H_L)/dx = wLp q_L^p + wLm q_L^m + wRp q_R^p + wRm q_R^m,
// and, with the face states q_L^m = q_{i-1} + s_{i-1}/2, q_L^p = q_i - s_i/2, q_R^m = q_i + s_i/2,
// q_R^p = q_{i+1} - s_{i+1}/2, every component costs its three slopes and seven multiply-adds:
//   (wLp + wRm) q_i + wLm q_{i-1} + wRp q_{i+1} + (wLm s_{i-1} + (wRm - wLp) s_i - wRp s_{i+1})/2.
template <typename R>
struct Faces {
  R c0, wLm, wRp, dW;    // c0 = wLp + wRm, dW = wRm - wLp
  R vpl_h, vmi_h;        // v^d at i+1 and i-1, times 1/(2 dx)
  int s;                 // element stride of direction d
};

// Root-find of one extrapolated face state (KT_IFACE_INVERT): f(e) = e - E + M^2/A = 0 with
// A = E + P0(e) + Pi, safeguarded Newton in the stencil precision inside [e_min, E] from `guess`;
// returns A at the root (v^d = M^d / A), or false if the state has none (E <= 0, M^2 >= E^2, no
// convergence in 100 steps).  FP64: stop at |de| <= 2^-50 E as the cell root-find; FP32: 2^-21 E.
template <typename R>
__device__ __forceinline__ bool face_root(const Params& P, R E, R M2, R Pi, R guess, R& A) {
  if (!(E > R(0)) || !(M2 < E * E) || !isfinite(E) || !isfinite(M2)) return false;
  if (!P.eos_table && (!P.bulk_on || Pi == R(0))) {
    const R M = sqrt(M2);  // conformal closed form, cancellation-free
    const R e = R(3) * (E - M) * (E + M) / (sqrt(fma(R(4) * E, E, R(-3) * M2)) + E);
    A = E + e * R(1.0 / 3.0) + Pi;
    return true;
  }
  R lo = (P.e_min > 0.0) ? R(P.e_min) : R(sizeof(R) == 8 ? 1e-300 : 1e-30), hi = E;
  R e = (guess >= lo && guess <= hi) ? guess : hi;
  const R stop = E * R(sizeof(R) == 8 ? 0x1p-50 : 0x1p-21);
  for (int it = 0; it < 100; ++it) {
    R p0, c2;
    eos_P_cs2<R>(P, e, p0, c2);
    A = E + p0 + Pi;
    const R f = e - E + M2 / A;
    if (f == R(0)) return true;
    if (f < R(0)) lo = e; else hi = e;
    R en = e - f / (R(1) - M2 * c2 / (A * A));
    if (!(en >= lo && en <= hi)) en = R(0.5) * (lo + hi);
    const R de = fabs(en - e);
    e = en;
    if (de <= stop) {
      if (e < R(P.e_min)) e = R(P.e_min);
      A = E + eos_P<R>(P, e) + Pi;
      return true;
    }
  }
  return false;
}

// KT_IFACE_INVERT (literal reading of Sec. 3.1): the four extrapolated states along D -- left face
// m (from cell i-1) and p (from cell i), right face m (from cell i) and p (from cell i+1) -- of the
// components the root-find reads (T^{tau mu}, pi^{tau mu}, Pi), each inverted from the e of the cell
// it was extrapolated from; v^d = M^d / (E + P0 + Pi) at the root, 0 for a state without one.
template <typename R, int D, bool TH1>
__device__ __forceinline__ void face_velocities_inverted(const Params& P, const Lattice& L, const StageIO<R>& io,
                                                         long long c, int s, R th, R gnn, R& vLm, R& vLp, R& vRm,
                                                         R& vRp) {
  const long long fs = L.fstride;
  const R h = R(0.5);
  R E4[4] = {R(0), R(0), R(0), R(0)}, M4[3][4] = {}, Pi4[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int n = (k < 8) ? k : 14;
    const R* p = io.qr_in + n * fs;
    const R a2 = ld<R>(p, c - 2 * s), a1 = ld<R>(p, c - s), a0 = ld<R>(p, c), b1 = ld<R>(p, c + s),
            b2 = ld<R>(p, c + 2 * s);
    const R d0 = a1 - a2, d1 = a0 - a1, d2 = b1 - a0, d3 = b2 - b1;
    R sm, s0, sp;
    three_slopes<R, TH1>(d0, d1, d2, d3, th, sm, s0, sp);
    const R x[4] = {fma(h, sm, a1), fma(-h, s0, a0), fma(h, s0, a0), fma(-h, sp, b1)};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (n == 0) E4[j] += x[j];
      else if (n == 4) E4[j] -= x[j];
      else if (n < 4) M4[n - 1][j] += x[j];
      else if (n < 8) M4[n - 5][j] -= x[j];
      else Pi4[j] = x[j];
    }
  }
  const R g[4] = {ld<R>(io.e_in, c - s), ld<R>(io.e_in, c), ld<R>(io.e_in, c), ld<R>(io.e_in, c + s)};
  R v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const R M2 = fma(M4[0][j], M4[0][j], fma(M4[1][j], M4[1][j], gnn * M4[2][j] * M4[2][j]));
    R A;
    v[j] = face_root<R>(P, E4[j], M2, Pi4[j], g[j], A) ? M4[D][j] / A : R(0);
  }
  vLm = v[0]; vLp = v[1]; vRm = v[2]; vRp = v[3];
}

// How the stencil reads u^mu around cell c: from the field arrays, through the read-only cache.
// (Staging u^mu in shared memory by TMA, like q, measured slower: the stencil's scattered u loads
// hit L1, which the larger shared-memory carve-out shrinks.)
template <typename R>
struct UGlobal {
  const R* u;
  long long fs, c;
  int sy, sz;  // row pitch, plane
  __device__ __forceinline__ R operator()(int m, int off) const { return ld<R>(u + m * fs, c + off); }
};
template <typename R>
__device__ __forceinline__ UGlobal<R> u_global(const Lattice& L, const StageIO<R>& io, long long c) {
  return UGlobal<R>{io.u_in, L.fstride, c, L.pitch, (int)L.plane};
}

// Velocity part of direction D: limited face states of u^tau and u^d and their ratio v^d
// (Sec. 3.1), the local speeds a = max(|v^p|, |v^m|) (Eq. ax), the central differences
// d_d u^mu and d_d v^d, and the pressure part of S_c (App. B):
// -d_d (v^d P delta^nu_tau - g^{d nu} P), P = P0 + Pi.
template <typename R, int D, bool TH1, bool IFACE, typename UA>
__device__ __forceinline__ void face_setup(const Params& P, const Lattice& L, const StageIO<R>& io, long long c,
                                           const UA& ua, const R (&uc)[4], R inv_gnn, R sfac, R (&dq)[NQ],
                                           R (&du)[4][4], R& dv, float& amax, Faces<R>& F) {
  const long long fs = L.fstride;
  const int s = (D == 0) ? 1 : ((D == 1) ? L.pitch : (int)L.plane);  // in the field arrays
  const int us = (D == 0) ? 1 : ((D == 1) ? ua.sy : ua.sz);           // where u is read
  const R hinv = pr<R>(P).half_inv_d[D];
  const R th = pr<R>(P).theta;

  R um1[4], up1[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    um1[m] = ua(m, -us);
    up1[m] = ua(m, us);
  }
  R vLm, vLp, vRm, vRp;
  if constexpr (IFACE) {
    face_velocities_inverted<R, D, TH1>(P, L, io, c, s, th, sfac * sfac, vLm, vLp, vRm, vRp);
  } else {
    const R u0t = uc[0], u0d = uc[D + 1];
    const R um2t = ua(0, -2 * us), um2d = ua(D + 1, -2 * us);
    const R up2t = ua(0, 2 * us), up2d = ua(D + 1, 2 * us);
    R t0 = um1[0] - um2t, t1 = u0t - um1[0], t2 = up1[0] - u0t, t3 = up2t - up1[0];
    R d0 = um1[D + 1] - um2d, d1 = u0d - um1[D + 1], d2 = up1[D + 1] - u0d, d3 = up2d - up1[D + 1];
    R st_m, st_0, st_p, sd_m, sd_0, sd_p;
    three_slopes<R, TH1>(t0, t1, t2, t3, th, st_m, st_0, st_p);
    three_slopes<R, TH1>(d0, d1, d2, d3, th, sd_m, sd_0, sd_p);
    const R h = R(0.5);
    vLm = vdiv(fma(h, sd_m, um1[D + 1]), fma(h, st_m, um1[0]));
    vLp = vdiv(fma(-h, sd_0, u0d), fma(-h, st_0, u0t));
    vRm = vdiv(fma(h, sd_0, u0d), fma(h, st_0, u0t));
    vRp = vdiv(fma(-h, sd_p, up1[D + 1]), fma(-h, st_p, up1[0]));
  }
  const R aL = nmax(fabs(vLp), fabs(vLm));
  const R aR = nmax(fabs(vRp), fabs(vRm));
  const R aF = nmax(aL, aR);  // both faces: the first cell's left face is nobody's right face
  amax = fmaxf(amax, to_f32((D == 2) ? aF * sfac : aF));
  const R wLp = (vLp - aL) * hinv, wRm = -(vRm + aR) * hinv;
  F.c0 = wLp + wRm;
  F.dW = wRm - wLp;
  F.wLm = (vLm + aL) * hinv;
  F.wRp = (aR - vRp) * hinv;

#pragma unroll
  for (int m = 0; m < 4; ++m) du[D + 1][m] = (up1[m] - um1[m]) * hinv;
  const R vpl = vdiv(up1[D + 1], up1[0]), vmi = vdiv(um1[D + 1], um1[0]);
  dv += (vpl - vmi) * hinv;
  F.vpl_h = vpl * hinv;
  F.vmi_h = vmi * hinv;
  F.s = s;

  const R* q = io.qr_in;
  const R Ppl = ld<R>(io.p_in, c + s) + ld<R>(q + 14 * fs, c + s);
  const R Pmi = ld<R>(io.p_in, c - s) + ld<R>(q + 14 * fs, c - s);
  dq[0] -= Ppl * F.vpl_h - Pmi * F.vmi_h;
  dq[D + 1] -= ((D == 2) ? (Ppl - Pmi) * inv_gnn : (Ppl - Pmi)) * hinv;
}

// row nu of T^{tau nu} that component n feeds through -d_d(-v^d pi^{tau nu}) (first == true:
// n = pi^{tau nu}) or -d_d(pi^{d nu}) (n = pi^{d nu}); -1 if none
template <int D>
__device__ __forceinline__ int cross_row(int n, bool first) {
  if (first) return (n >= 4 && n <= 7) ? n - 4 : -1;
#pragma unroll
  for (int nu = 0; nu < 4; ++nu)
    if (n == pix(D + 1, nu)) return nu;
  return -1;
}

// dq[r] += v for a warp-uniform runtime row r (the switch keeps dq in registers)
template <typename R>
__device__ __forceinline__ void add_row(R (&dq)[NQ], int r, R v) {
  switch (r) {
    case 0: dq[0] += v; break;
    case 1: dq[1] += v; break;
    case 2: dq[2] += v; break;
    case 3: dq[3] += v; break;
    case 4: dq[4] += v; break;
    case 5: dq[5] += v; break;
    case 6: dq[6] += v; break;
    case 7: dq[7] += v; break;
    case 8: dq[8] += v; break;
    case 9: dq[9] += v; break;
    case 10: dq[10] += v; break;
    case 11: dq[11] += v; break;
    case 12: dq[12] += v; break;
    case 13: dq[13] += v; break;
    case 14: dq[14] += v; break;
    default: break;
  }
}

// one component along one direction: generalised-minmod reconstruction from the five-point
// stencil p[-2s..2s] (a0 = p[0] given; global memory, or shared memory if SMEM) and the flux
// difference -(H_R - H_L)/dx, added to acc; a1, b1 return the neighbours for the central
// differences of S_c
template <typename R, bool SMEM, bool TH1 = false>
__device__ __forceinline__ R component_flux(const R* p, int s, R a0, R th, const Faces<R>& F, R& a1, R& b1, R acc) {
  R a2, b2;
  if constexpr (SMEM) {
    a2 = p[-2 * s]; a1 = p[-s]; b1 = p[s]; b2 = p[2 * s];
  } else {
    a2 = ld<R>(p, -2 * s); a1 = ld<R>(p, -s); b1 = ld<R>(p, s); b2 = ld<R>(p, 2 * s);
  }
  const R d0 = a1 - a2, d1 = a0 - a1, d2 = b1 - a0, d3 = b2 - b1;
  R sm, s0, sp;
  three_slopes<R, TH1>(d0, d1, d2, d3, th, sm, s0, sp);
  const R slopes = fma(F.wLm, sm, fma(F.dW, s0, -F.wRp * sp));
  acc = fma(F.c0, a0, acc);
  acc = fma(F.wLm, a1, acc);
  acc = fma(F.wRp, b1, acc);
  return fma(R(0.5), slopes, acc);
}

// Component n (warp-uniform) of the 15 conserved components, at a cell whose stencil starts at
// p with strides sx, sy, sz: -div H in x, y, eta and the remaining S_c terms
// -d_d(-v^d pi^{tau nu} + pi^{d nu}) by central differences, added to dq.
template <typename R, bool SMEM, bool TH1 = false>
__device__ __forceinline__ void component_rhs(const Params& P, int n, const R* p, int sx, int sy, int sz, R th,
                                              const Faces<R>& Fx, const Faces<R>& Fy, const Faces<R>& Fz,
                                              R (&dq)[NQ]) {
  const R a0 = SMEM ? p[0] : ld<R>(p, 0);
  R a1x, b1x, a1y, b1y, a1z, b1z;
  R acc = component_flux<R, SMEM, TH1>(p, sx, a0, th, Fx, a1x, b1x, R(-0.0));
  acc = component_flux<R, SMEM, TH1>(p, sy, a0, th, Fy, a1y, b1y, acc);
  acc = component_flux<R, SMEM, TH1>(p, sz, a0, th, Fz, a1z, b1z, acc);
  add_row(dq, n, acc);
  if (n >= 4 && n <= 13) {  // pi components
    const int r0 = cross_row<0>(n, true);
    if (r0 >= 0)
      add_row(dq, r0, (Fx.vpl_h * b1x - Fx.vmi_h * a1x) + (Fy.vpl_h * b1y - Fy.vmi_h * a1y) +
                          (Fz.vpl_h * b1z - Fz.vmi_h * a1z));
    const int rx = cross_row<0>(n, false), ry = cross_row<1>(n, false), rz = cross_row<2>(n, false);
    const R* hinv = pr<R>(P).half_inv_d;  // kernel parameters: no registers held across the loop
    if (rx >= 0) add_row(dq, rx, -(b1x - a1x) * hinv[0]);
    if (ry >= 0) add_row(dq, ry, -(b1y - a1y) * hinv[1]);
    if (rz >= 0) add_row(dq, rz, -(b1z - a1z) * hinv[2]);
  }
}

// ---- paired FP32 arithmetic (the f32x2 instructions of the sm_100 family): two independent
// single-precision operations, each rounded to nearest as its scalar form, in one instruction
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void up2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// The x and y face weights of a cell as (x, y) pairs for the paired flux of component_rhs_xy.
struct FacesXY {
  unsigned long long c0, wLm, dW, nwRp, wRp;
};
__device__ __forceinline__ FacesXY faces_xy(const Faces<float>& Fx, const Faces<float>& Fy) {
  return FacesXY{pk2(Fx.c0, Fy.c0), pk2(Fx.wLm, Fy.wLm), pk2(Fx.dW, Fy.dW), pk2(-Fx.wRp, -Fy.wRp), pk2(Fx.wRp, Fy.wRp)};
}

// component_rhs for the FP32 stencil in shared memory with theta = 1, the x and y directions
// computed as pairs: the differences, the slope combination and the seven multiply-adds of the
// two directions share instructions; the limiter's min/max and the eta direction stay scalar.
// The same arithmetic as component_rhs, summed x + y, then eta.
__device__ __forceinline__ void component_rhs_xy(const Params& P, int n, const float* p, int sy, int sz,
                                                 const FacesXY& W, const Faces<float>& Fx, const Faces<float>& Fy,
                                                 const Faces<float>& Fz, float (&dq)[NQ]) {
  const float a0 = p[0];
  const float a2x = p[-2], a1x = p[-1], b1x = p[1], b2x = p[2];
  const float a2y = p[-2 * sy], a1y = p[-sy], b1y = p[sy], b2y = p[2 * sy];
  const unsigned long long A0 = pk2(a0, a0), A1 = pk2(a1x, a1y), B1 = pk2(b1x, b1y);
  const unsigned long long D0 = sub2(A1, pk2(a2x, a2y)), D1 = sub2(A0, A1), D2 = sub2(B1, A0),
                           D3 = sub2(pk2(b2x, b2y), B1);
  float d0x, d0y, d1x, d1y, d2x, d2y, d3x, d3y, smx, smy, s0x, s0y, spx, spy;
  up2(D0, d0x, d0y);
  up2(D1, d1x, d1y);
  up2(D2, d2x, d2y);
  up2(D3, d3x, d3y);
  three_slopes<float, true>(d0x, d1x, d2x, d3x, 1.f, smx, s0x, spx);
  three_slopes<float, true>(d0y, d1y, d2y, d3y, 1.f, smy, s0y, spy);
  const unsigned long long slopes = fma2(W.wLm, pk2(smx, smy), fma2(W.dW, pk2(s0x, s0y), mul2(W.nwRp, pk2(spx, spy))));
  unsigned long long acc = mul2(W.c0, A0);
  acc = fma2(W.wLm, A1, acc);
  acc = fma2(W.wRp, B1, acc);
  acc = fma2(pk2(0.5f, 0.5f), slopes, acc);
  float accx, accy, a1z, b1z;
  up2(acc, accx, accy);
  const float accz = component_flux<float, true, true>(p, sz, a0, 1.f, Fz, a1z, b1z, accx + accy);
  add_row(dq, n, accz);
  if (n >= 4 && n <= 13) {  // pi components
    const int r0 = cross_row<0>(n, true);
    if (r0 >= 0)
      add_row(dq, r0, (Fx.vpl_h * b1x - Fx.vmi_h * a1x) + (Fy.vpl_h * b1y - Fy.vmi_h * a1y) +
                          (Fz.vpl_h * b1z - Fz.vmi_h * a1z));
    const int rx = cross_row<0>(n, false), ry = cross_row<1>(n, false), rz = cross_row<2>(n, false);
    const float* hinv = pr<float>(P).half_inv_d;
    if (rx >= 0) add_row(dq, rx, -(b1x - a1x) * hinv[0]);
    if (ry >= 0) add_row(dq, ry, -(b1y - a1y) * hinv[1]);
    if (rz >= 0) add_row(dq, rz, -(b1z - a1z) * hinv[2]);
  }
}

// All 15 components from global memory.  The component loop is not unrolled: one compact body
// keeps the instruction stream of the whole kernel small.
template <typename R, bool TH1 = false>
__device__ __forceinline__ void conserved_fluxes(const Params& P, const Lattice& L, const StageIO<R>& io, long long c,
                                                 const Faces<R>& Fx, const Faces<R>& Fy, const Faces<R>& Fz,
                                                 R (&dq)[NQ]) {
  const long long fs = L.fstride;
  const R th = pr<R>(P).theta;
  const R* p = io.qr_in + c;
#pragma unroll 1
  for (int n = 0; n < NQ; ++n, p += fs) component_rhs<R, false, TH1>(P, n, p, Fx.s, Fy.s, Fz.s, th, Fx, Fy, Fz, dq);
}

// ------------------------------------------------------------- d) the root-find (Sec. 2.4)
// Positive doubles are ordered like their bit patterns read as integers, so the brackets and
// tolerances below are compared with integer instructions and the slow FP64 pipe only does
// arithmetic.
__device__ __forceinline__ long long obits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ long long abits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }
__device__ __forceinline__ double clamp_pos(double x, double lo, double hi) {  // lo, hi > 0; NaN -> hi
  return (obits(x) < obits(lo)) ? lo : ((obits(x) <= obits(hi)) ? x : hi);
}

// The interval of e > 0 in the FP64 table and its record: the single-precision log guess of
// eos_interval, checked against both ends of the interval in the same load; only a guess that
// misses (next to a node) searches as eos_interval does (integer comparisons of the bit patterns)
// and loads again.  The same interval as eos_interval, with one dependent load instead of three.
// Seg is RootSeg (FP64 path) or RootSegM (mixed precision); both start with e0, e1.
__device__ __forceinline__ RootSeg load_root_seg(const RootSeg* p) {
  const double2* d = reinterpret_cast<const double2*>(p);
  const double2 v0 = __ldg(d), v1 = __ldg(d + 1), v2 = __ldg(d + 2);
  const float4 v3 = __ldg(reinterpret_cast<const float4*>(p) + 3);
  return RootSeg{v0.x, v0.y, v1.x, v1.y, v2.x, v2.y, v3.x, v3.y, v3.z, v3.w};
}
__device__ __forceinline__ RootSegM load_root_seg(const RootSegM* p) {
  const double2* d = reinterpret_cast<const double2*>(p);
  const double2 v0 = __ldg(d), v1 = __ldg(d + 1);
  const float4 v2 = __ldg(reinterpret_cast<const float4*>(p) + 2);
  const float b3 = __ldg(reinterpret_cast<const float*>(p) + 12);
  return RootSegM{v0.x, v0.y, v1.x, v1.y, v2.x, v2.y, v2.z, v2.w, b3, 0.f, 0.f, 0.f};
}
template <typename Seg>
__device__ __forceinline__ Seg root_seg(const Params& P, const Seg* seg, double e) {
  const int n1 = P.eos_n - 2;
  const float g = (__logf(d2f_trunc(e)) - P.lne0) * P.inv_h;
  int i = min((g > 0.f) ? (int)g : 0, n1);  // NaN compares false -> 0
  const long long b = obits(e);
  Seg s = load_root_seg(seg + i);
  if ((i > 0 && b < obits(s.e0)) || b >= obits(s.e1)) {
#pragma unroll 1
    for (int it = 0; it < 64 && i > 0 && b < obits(seg[i].e0); ++it) --i;
#pragma unroll 1
    for (int it = 0; it < 64 && i < n1 && b >= obits(seg[i].e1); ++it) ++i;
    s = load_root_seg(seg + i);
  }
  return s;
}

// the interval's record for the FP64 path (RootSeg) or the mixed-precision one (RootSegM)
template <bool MIXED>
__device__ __forceinline__ auto path_seg(const Params& P, double e) {
  if constexpr (MIXED) return root_seg(P, P.seg_m, e);
  else return root_seg(P, P.seg_r, e);
}

// P0(e) in d = e - e0 on the interval's record: the cubic in FP64 (RootSeg), or (RootSegM) its
// leading part in FP64 with the correction d (a2 + d a3) to a1 formed in single precision from
// df, the single-precision d.
__device__ __forceinline__ double seg_P(const RootSeg& s, double d, float) {
  return fma(d, fma(d, fma(d, s.a3, s.a2), s.a1), s.P0);
}
__device__ __forceinline__ double seg_P(const RootSegM& s, double d, float df) {
  return fma(d, s.a1 + f2d_bits(df * fmaf(df, s.a3, s.a2)), s.P0);
}

// The residual in product form g(e) = (e - E) A(e) + M^2 = f(e) A(e), A = E + P0(e) + Pi > 0:
// the root and the sign of f(e) = e - E + M^2 / A of Eq. (eInferred), without a reciprocal.
// Also A, P0(e) and, in single precision, A (truncated) and A f'(e) = A - M^2 c_s^2 / A: the
// Newton step on f, e - f/f' = e - g/(A f'), then needs the FP64 product of g with a
// single-precision factor (which only sets the step length; f is nearly linear in e where M is
// small, g is not).  MIXED: P0 from the mixed-precision records (RootSegM), whose rounding of the
// cubic's correction term (~1e-13 of P0, in steps as d crosses single-precision values) is far
// below the learned start's 1e-10 acceptance but above the plain root-find's 2^-50 stop, so only
// the learned start's Newton steps use it.
struct Resid {
  double g, A, p0;
  float gp, Af;
};
template <bool MIXED>
__device__ __forceinline__ Resid residual(const Params& P, double e, double E, double EPi, double M2, float M2f) {
  const auto s = path_seg<MIXED>(P, e);
  const double d = e - s.e0;
  const float df = d2f_trunc(d);
  Resid r;
  r.p0 = seg_P(s, d, df);
  r.A = EPi + r.p0;
  const double em = e - E;
  r.g = fma(em, r.A, M2);
  const float c2 = fmaf(df, fmaf(df, s.b3, s.b2), s.b1);
  r.Af = d2f_trunc(r.A);
  r.gp = r.Af - __fdividef(M2f * c2, r.Af);
  return r;
}

// one Newton step on f: e - g / (A f')
__device__ __forceinline__ double newton_step(double e, const Resid& r) {
  return fma(-r.g, f2d_bits(__frcp_rn(r.gp)), e);
}

// P0(e) on the FP64 table
__device__ __forceinline__ double eos_P_pos(const Params& P, double e) {
  const RootSeg s = root_seg(P, P.seg_r, e);
  return seg_P(s, e - s.e0, 0.f);
}

// Plain root-find: safeguarded Newton inside the bracket [e_min, E] (a step that leaves it
// bisects), from `start` if it lies inside, else from E; stop at |de| <= 2^-50 E (g is known to
// about one ulp of E A), at most 100 steps.  Table EOS only.  The stop's bit pattern is E's with
// the exponent lowered by 50 (exact for E >= 2^-972; smaller E stops only at de = 0).
__device__ __forceinline__ unsigned rootfind_plain(const Params& P, double E, double EPi, double M2, float M2f,
                                                   double start, double& e, double& P0, unsigned& iters) {
  double lo = (P.e_min > 0.0) ? P.e_min : 1e-300, hi = E;
  e = (obits(start) >= obits(lo) && obits(start) <= obits(hi)) ? start : hi;
  const long long stop = max(obits(E) - (50LL << 52), 0LL);
  int it;
  for (it = 0; it < 100; ++it) {
    const Resid r = residual<false>(P, e, E, EPi, M2, M2f);
    if (abits(r.g) == 0) break;
    if (obits(r.g) < 0) lo = e; else hi = e;
    double en = newton_step(e, r);
    if (!(obits(en) >= obits(lo) && obits(en) <= obits(hi))) en = 0.5 * (lo + hi);
    const double de = en - e;
    e = en;
    if (abits(de) <= stop) { ++it; break; }
  }
  iters += (unsigned)it;
  if (obits(e) < obits(P.e_min)) e = P.e_min;
  P0 = eos_P_pos(P, e);
  return (it >= 100) ? ST_INVERSION : 0u;
}

// ------------------------------------------------------------ d) inversion, FP64 (Sec. 2.4)
// T^{tau mu} -> (e, P0, u^mu) at tau (Eqs. eInferred-uiInferred): the safeguarded Newton of
// rootfind_plain from the cell's previous e; with the conformal EOS and no bulk pressure, the
// closed form.
__device__ __forceinline__ unsigned invert_fp64(const Params& P, double tau, const double (&qn)[NQ], double guess,
                                                double& e, double& P0, double (&uo)[4], unsigned& iters) {
  const double E = qn[0] - qn[4];
  const double Mx = qn[1] - qn[5], My = qn[2] - qn[6], Mn = qn[3] - qn[7];
  const double Pi = qn[14];
  const double gnn = P.milne ? tau * tau : 1.0;
  const double M2 = fma(Mx, Mx, fma(My, My, gnn * Mn * Mn));
  unsigned st = 0;
  if (!(E > 0.0) || !isfinite(E) || !isfinite(M2) || !(M2 < E * E)) {
    st = ST_INVERSION;
    e = (P.e_min > 0.0) ? P.e_min : 1e-30;
    P0 = eos_P<double>(P, e);
  } else if (!P.eos_table) {  // (bulk pressure is evolved with a table EOS only)
    const double M = sqrt(M2);  // conformal closed form e = sqrt(4E^2 - 3M^2) - E, cancellation-free
    e = 3.0 * (E - M) * (E + M) / (sqrt(fma(4.0 * E, E, -3.0 * M2)) + E);
    if (e < P.e_min) e = P.e_min;
    P0 = e * (1.0 / 3.0);
  } else {
    st = rootfind_plain(P, E, E + Pi, M2, d2f_trunc(M2), guess, e, P0, iters);
  }
  if (st) {
    uo[0] = 1.0; uo[1] = uo[2] = uo[3] = 0.0;
  } else {
    const double Pt = P0 + Pi;
    const double ut = sqrt(vdiv(E + Pt, e + Pt));
    const double w = vdiv(1.0, (e + Pt) * ut);
    uo[0] = ut; uo[1] = Mx * w; uo[2] = My * w; uo[3] = Mn * w;
  }
  if (!isfinite(e) || !isfinite(uo[0]) || !isfinite(uo[1]) || !isfinite(uo[2]) || !isfinite(uo[3]))
    st |= ST_NONFINITE;
  return st;
}

// ------------------------------------------------------------ e) regulator (Sec. 3.2)
template <typename R>
__device__ __forceinline__ R regulator_factor(const Params& P, R gnn, R e, R P0, const R (&u)[4], const R (&pi)[4][4],
                                              R Pi) {
  const R glo[4] = {R(1), R(-1), R(-1), -gnn};
  const R gup[4] = {R(1), R(-1), R(-1), -sdiv(R(1), gnn)};
  R PP = R(-0.0);  // -0 is the exact additive identity (x + -0 = x), so zero terms fold away
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      R X = Pi * (((a == b) ? gup[a] : R(-0.0)) - u[a] * u[b]) + pi[a][b];
      PP += X * X * glo[a] * glo[b];
    }
  if (!(PP > R(0))) return R(1);
  R nPP = sqrt(PP);
  R rho = sdiv(nPP, pr<R>(P).rho_max * sqrt(e * e + R(3) * P0 * P0));
  R den = sdiv(R(1), pr<R>(P).xi0_rho_max * nPP);
  R tr = pi[0][0] - pi[1][1] - pi[2][2] - gnn * pi[3][3];
  rho = nmax(rho, fabs(tr) * den);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    R o = pi[l][0] * u[0] - pi[l][1] * u[1] - pi[l][2] * u[2] - gnn * pi[l][3] * u[3];
    if (l == 3 && P.milne) o *= sqrt(gnn);
    rho = nmax(rho, fabs(o) * den);
  }
  if (rho < R(1e-4)) return R(1) - rho * rho * R(1.0 / 3.0);
  return sdiv(tanh(rho), rho);
}

// ---------------------------------------------------------------- f) stores with ghosts
template <typename R>
__device__ __forceinline__ void store_cell(const StageIO<R>& io, long long fs, long long t, const double (&qn)[NQ],
                                           const R (&qr)[NQ], const R (&uo)[4], R e, R P0) {
#pragma unroll
  for (int n = 0; n < NQ; ++n) io.q_out[n * fs + t] = qn[n];
  if (io.qr_out) {
#pragma unroll
    for (int n = 0; n < NQ; ++n) io.qr_out[n * fs + t] = qr[n];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) io.u_out[m * fs + t] = uo[m];
  io.e_out[t] = e;
  io.p_out[t] = P0;
}

// padded ghost coordinate g in {0, 1, n+2, n+3} that copies the physical padded coordinate p
__device__ __forceinline__ int ghost_source(int g, int n, int periodic) {
  if (periodic) return 2 + (((g - 2) % n) + n) % n;
  return (g < 2) ? 2 : n + 1;
}

// calls put(t) for the element index t of the padded cell (i, j, k) and of every ghost cell that
// copies it (Eqs. ghostCells_1/2, or the periodic images)
template <typename F>
__device__ __forceinline__ void for_cell_and_ghosts(const Params& P, const Lattice& L, int i, int j, int k, F&& put) {
  put(L.idx(i, j, k));
  const int nn[3] = {L.nx, L.ny, L.nz};
  const int pc[3] = {i, j, k};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    int n = nn[ax];
    if (pc[ax] > 3 && pc[ax] < n) continue;  // interior cells own no ghost
    const int gs[4] = {0, 1, n + 2, n + 3};
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (ghost_source(gs[g], n, P.periodic) != pc[ax]) continue;
      int ii = (ax == 0) ? gs[g] : i, jj = (ax == 1) ? gs[g] : j, kk = (ax == 2) ? gs[g] : k;
      put(L.idx(ii, jj, kk));
    }
  }
}

template <typename R>
__device__ __forceinline__ void store_with_ghosts(const Params& P, const Lattice& L, const StageIO<R>& io, int i,
                                                  int j, int k, const double (&qn)[NQ], const R (&qr)[NQ],
                                                  const R (&uo)[4], R e, R P0) {
  const long long fs = L.fstride;
  for_cell_and_ghosts(P, L, i, j, k, [&](long long t) { store_cell<R>(io, fs, t, qn, qr, uo, e, P0); });
}

// ---------------------------------------------------------------- a) + b) for one cell
// dq = C[q] of Eq. (semiDiscreteKT) at the cell c: -div H in x, y, eta plus the source vector
// J = S + G (App. B), in the stencil precision R, evaluated at tau.  In three parts: the cell's
// face data (velocities, speeds, flux weights, d_d u^mu, d_i v^i, pressure part of S_c), the 15
// components' fluxes (conserved_fluxes or a shared-memory loop), then the sources.
template <typename R>
struct CellGeom {
  R tau, gnn, inv_gnn;
};
template <typename R>
__device__ __forceinline__ CellGeom<R> cell_geom(const Params& P, double tau_src) {
  CellGeom<R> g;
  g.tau = from_f64<R>(tau_src);
  g.gnn = P.milne ? g.tau * g.tau : R(1);
  g.inv_gnn = P.milne ? sdiv(R(1), g.gnn) : R(1);
  return g;
}

// the three directions' face setups; uc returns u^mu at the cell
template <typename R, bool TH1, bool IFACE, typename UA>
__device__ __forceinline__ void cell_faces(const Params& P, const Lattice& L, const StageIO<R>& io, long long c,
                                           const UA& ua, const CellGeom<R>& G, R (&dq)[NQ], R (&uc)[4],
                                           R (&du)[4][4], R& dv, float& amax, Faces<R>& Fx, Faces<R>& Fy,
                                           Faces<R>& Fz) {
#pragma unroll
  for (int n = 0; n < NQ; ++n) dq[n] = R(-0.0);  // exact additive identity
#pragma unroll
  for (int m = 0; m < 4; ++m) uc[m] = ua(m, 0);
  dv = R(-0.0);
  const R sfac = P.milne ? G.tau : R(1);  // sqrt(-g_{eta eta}): speeds along eta in units of c
  face_setup<R, 0, TH1, IFACE>(P, L, io, c, ua, uc, G.inv_gnn, sfac, dq, du, dv, amax, Fx);
  face_setup<R, 1, TH1, IFACE>(P, L, io, c, ua, uc, G.inv_gnn, sfac, dq, du, dv, amax, Fy);
  face_setup<R, 2, TH1, IFACE>(P, L, io, c, ua, uc, G.inv_gnn, sfac, dq, du, dv, amax, Fz);
}

template <typename R, bool DIAG = false>
__device__ __forceinline__ void cell_sources(const Params& P, const Lattice& L, const StageIO<R>& io, long long c,
                                             const CellGeom<R>& G, const R (&uc)[4], R (&du)[4][4], R dv,
                                             R (&dq)[NQ], R* dg = nullptr);

template <typename R, bool TH1 = false, bool IFACE = false>
__device__ __forceinline__ void cell_rhs(const Params& P, const Lattice& L, const StageIO<R>& io, long long c,
                                         double tau_src, R (&dq)[NQ], float& amax) {
  const CellGeom<R> G = cell_geom<R>(P, tau_src);
  R uc[4], du[4][4];
  R dv;
  Faces<R> Fx, Fy, Fz;
  cell_faces<R, TH1, IFACE>(P, L, io, c, u_global(L, io, c), G, dq, uc, du, dv, amax, Fx, Fy, Fz);
  conserved_fluxes<R, TH1>(P, L, io, c, Fx, Fy, Fz, dq);
  cell_sources<R>(P, L, io, c, G, uc, du, dv, dq);
}

// The source vector J = S + G of App. B at the cell, added to dq.  DIAG: also the validity
// diagnostics of Sec. 7 into dg[0..5]: tau_pi theta, tau_Pi theta (unfloored relaxation times),
// sqrt(pi.pi)/P0, |Pi|/P0, sqrt(J^{mu nu} J_{mu nu})/(2 eta sqrt(sigma.sigma)) and |J|/(zeta
// |theta|) with J^{mu nu}, J the second-order terms of Eq. (14_moment_terms) (no diffusion); a
// quantity whose channel is off, or whose denominator vanishes, is 0.
template <typename R, bool DIAG>
__device__ __forceinline__ void cell_sources(const Params& P, const Lattice& L, const StageIO<R>& io, long long c,
                                             const CellGeom<R>& G, const R (&uc)[4], R (&du)[4][4], R dv,
                                             R (&dq)[NQ], R* dg) {
  if constexpr (DIAG) {
#pragma unroll
    for (int k = 0; k < 6; ++k) dg[k] = R(0);
  }
  const long long fs = L.fstride;
  const R tau = G.tau, gnn = G.gnn, inv_gnn = G.inv_gnn;
  // ---- b) sources at the cell
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    du[0][m] = (uc[m] - ld<R>(io.u_prev + m * fs, c)) * pr<R>(P).inv_dtau;  // backward difference
  }
  const R* q = io.qr_in;
  R pi[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) {
      pi[a][b] = ld<R>(q + pix(a, b) * fs, c);
      pi[b][a] = pi[a][b];
    }
  const R Pic = ld<R>(q + 14 * fs, c);
  const R ec = ld<R>(io.e_in, c), P0c = ld<R>(io.p_in, c);
  const R Pt = P0c + Pic;
  const R it = P.milne ? tau * inv_gnn : R(0);  // Gamma^eta_{tau eta} = 1/tau
  const R tg = P.milne ? tau : R(0);         // Gamma^tau_{eta eta}

  // geometric sources of the conservation laws, Eqs. (dT001)-(dT0i1)
  {
    R Tnn = (ec + Pt) * uc[3] * uc[3] + Pt * inv_gnn + pi[3][3];
    dq[0] -= ld<R>(q, c) * it + tg * Tnn;
    dq[1] -= ld<R>(q + fs, c) * it;
    dq[2] -= ld<R>(q + 2 * fs, c) * it;
    dq[3] -= R(3) * ld<R>(q + 3 * fs, c) * it;
  }

  if (P.shear_on || P.bulk_on) {
    const R glo[4] = {R(1), R(-1), R(-1), -gnn};
    const R gup[4] = {R(1), R(-1), R(-1), -inv_gnn};
    // u^mu_{;alpha}, alpha = 0..3 (only Gamma^eta_{tau eta} = 1/tau, Gamma^tau_{eta eta} = tau)
    R cov[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      cov[0][a] = du[a][0] + ((a == 3) ? tg * uc[3] : R(-0.0));
      cov[1][a] = du[a][1];
      cov[2][a] = du[a][2];
      cov[3][a] = du[a][3] + ((a == 0) ? it * uc[3] : ((a == 3) ? it * uc[0] : R(-0.0)));
    }
    const R theta = cov[0][0] + cov[1][1] + cov[2][2] + cov[3][3];
    const R theta3 = theta * R(1.0 / 3.0);
    R Dup[4], Dlo[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      Dup[m] = uc[0] * cov[m][0] + uc[1] * cov[m][1] + uc[2] * cov[m][2] + uc[3] * cov[m][3];
      Dlo[m] = glo[m] * Dup[m];
    }
    // nabla^a u^m = Delta^{a b} u^m_{;b} = g^{aa} u^m_{;a} - u^a D u^m
    R nab[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int m = 0; m < 4; ++m) nab[a][m] = gup[a] * cov[m][a] - uc[a] * Dup[m];
    R sig[4][4], om[4][4];  // symmetric and antisymmetric: each pair is computed once
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a; b < 4; ++b) {
        R Dab = ((a == b) ? gup[a] : R(-0.0)) - uc[a] * uc[b];
        sig[a][b] = R(0.5) * (nab[a][b] + nab[b][a]) - theta3 * Dab;
        sig[b][a] = sig[a][b];
        om[a][b] = (a == b) ? R(0) : R(0.5) * (nab[b][a] - nab[a][b]);  // App. A convention
        om[b][a] = -om[a][b];
      }
    R ps = R(-0.0);  // pi^{mu nu} sigma_{mu nu}
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) ps += pi[a][b] * sig[a][b] * glo[a] * glo[b];
    const R ps3 = ps * R(1.0 / 3.0);

    // transport coefficients (Sec. 2.2) from T(e), ln(1/3 - c_s^2)(e)
    R T, lnd;
    eos_T_lnd<R>(P, ec, T, lnd);
    const R iu0 = sdiv(R(1), uc[0]);

    if (P.shear_on) {
      R eta_tp = (ec + P0c) * R(0.2);
      R es = eta_over_s<R>(P, T);
      R rate_pi = (es > R(0)) ? sdiv(T, R(5) * es) : R(INFINITY);
      rate_pi = fmin(rate_pi, pr<R>(P).rate_max);
      const R tpp = pr<R>(P).tpp;
      R xs = R(-0.0);  // sigma.sigma (diagnostics)
      R av[4];  // pi^{mu lambda} D u_lambda
#pragma unroll
      for (int m = 0; m < 4; ++m) av[m] = pi[m][0] * Dlo[0] + pi[m][1] * Dlo[1] + pi[m][2] * Dlo[2] + pi[m][3] * Dlo[3];
      // B^{mu nu} = pi^{mu l} g_ll omega^{nu l};  C^{mu nu} = pi^{mu l} g_ll sigma^{nu l}
      R B[4][4], Cm[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          R sb = R(-0.0), sc = R(-0.0);
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            if (l != b) sb += pi[a][l] * glo[l] * om[b][l];  // omega^{bb} = 0
            sc += pi[a][l] * glo[l] * sig[b][l];
          }
          B[a][b] = sb;
          Cm[a][b] = sc;
        }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
          R Dab = ((a == b) ? gup[a] : R(-0.0)) - uc[a] * uc[b];
          R I1 = av[a] * uc[b] + av[b] * uc[a];
          R I3 = B[a][b] + B[b][a];
          R I4 = R(0.5) * (Cm[a][b] + Cm[b][a]) - Dab * ps3;
          R Ipi = I1 + R(4.0 / 3.0) * theta * pi[a][b] - I3 + tpp * I4 - R(1.2) * Pic * sig[a][b];
          R S = (R(2) * eta_tp * sig[a][b] - rate_pi * pi[a][b] - Ipi) * iu0 + pi[a][b] * dv;
          if constexpr (DIAG) {  // sums over the full tensor: off-diagonal pairs count twice
            const R w = glo[a] * glo[b] * ((a == b) ? R(1) : R(2));
            const R X = Ipi - I1;  // -J^{ab}/tau_pi
            dg[2] += pi[a][b] * pi[a][b] * w;
            dg[4] += X * X * w;
            xs += sig[a][b] * sig[a][b] * w;
          }
          // -G^{ab}/u^tau with G^{ab} = u^c Gamma^a_{cd} pi^{db} + (a <-> b)
          R ha = (a == 0) ? tg * uc[3] * pi[3][b] : ((a == 3) ? it * (uc[0] * pi[3][b] + uc[3] * pi[0][b]) : R(-0.0));
          R hb = (b == 0) ? tg * uc[3] * pi[3][a] : ((b == 3) ? it * (uc[0] * pi[3][a] + uc[3] * pi[0][a]) : R(-0.0));
          const bool geo = (a == 0 || a == 3 || b == 0 || b == 3);  // (a, b) in {1, 2}^2: G^{ab} = 0
          dq[pix(a, b)] += geo ? S - (ha + hb) * iu0 : S;
        }
      if constexpr (DIAG) {
        dg[0] = sdiv(R(5) * es, T) * theta;
        dg[4] = (xs > R(0)) ? sdiv(sqrt(dg[4]), R(2) * eta_tp * sqrt(xs)) : R(0);
        (void)xs;
      }
    }
    if (P.bulk_on) {
      R lrate = R(2.70805020110221) + R(2) * lnd + slog(T) - ln_zeta_over_s<R>(P, T);  // ln 15 + ...
      R rate_Pi = fmin(sexp(lrate), pr<R>(P).rate_max);
      R d = sexp(lnd);
      R zt = R(15) * d * d * (ec + P0c);
      R IPi = R(2.0 / 3.0) * Pic * theta - R(1.6) * d * ps;
      dq[14] += (-zt * theta - rate_Pi * Pic - IPi) * iu0 + Pic * dv;
      if constexpr (DIAG) {
        dg[1] = sexp(-lrate) * theta;
        dg[5] = (theta != R(0)) ? sdiv(fabs(IPi), zt * fabs(theta)) : R(0);
      }
    }
    if constexpr (DIAG) {
      dg[2] = sdiv(sqrt(dg[2]), P0c);
      dg[3] = sdiv(fabs(Pic), P0c);
    }
  }
}

// The inversion's inputs at one cell (Eqs. eInferred-uiInferred): E = T^tt - pi^tt,
// M^i = T^ti - pi^ti, Pi and M^2 = M_x^2 + M_y^2 + g_nn M_n^2 in FP64; E and M^2 also truncated to
// single precision for the network's features, the Newton step factor and the quick test of
// M^2 < E^2.
struct InvIn {
  double E, Mx, My, Mn, Pi, M2;
  float Ef, M2f;
};
__device__ __forceinline__ InvIn inv_in(double gnn, double E, double Mx, double My, double Mn, double Pi) {
  InvIn v;
  v.E = E; v.Mx = Mx; v.My = My; v.Mn = Mn; v.Pi = Pi;
  v.M2 = fma(gnn * Mn, Mn, fma(My, My, Mx * Mx));
  v.Ef = d2f_trunc(E);
  v.M2f = d2f_trunc(v.M2);
  return v;
}

// The network's start for the root-find of the inversion inputs v: the conformal root corrected
// by y = r^2 z (r^2 = M^2/E^2, feature 1), e = E (e_conf/E) exp(y/10), with z the network's
// output for this cell at the start of the step (mlp_start_kernel).  The correction vanishes at
// rest, where e_conf = E is the root, and the network's BF16 error scales with it; cells with
// r^2 <= kMlpGateR2 start from e_conf.
__device__ __forceinline__ double learned_start(const InvIn& v, float z) {
  float x[MLP_IN], ecE;
  mlp_features(fmaxf(v.Ef, 1e-30f), v.M2f, d2f_trunc(v.Pi), x, ecE);
  const float y = (x[1] > kMlpGateR2) ? x[1] * z : 0.f;
  return f2d_bits(v.Ef * ecE * __expf(0.1f * y));
}

// ---------------------------------------------------------------- one cell of a tile (FP64)
// The whole stage for one cell in one thread; cells past the edge of the event (valid = false)
// compute nothing and store nothing.
template <typename R, int STAGE, bool TH1, bool IFACE>
__device__ __forceinline__ void stage_cell(const Params& P, const Lattice& L, const StageIO<R>& io, int i, int j,
                                           int k, unsigned& st, unsigned& nit, unsigned& nreg, float& amax) {
  static_assert(sizeof(R) == 8, "the fused stage is the FP64 path; mixed precision uses kt_split.cuh");
  const bool valid = (i < L.nx) && (j < L.ny) && (k < L.nz);
  const long long fs = L.fstride;
  const long long c = L.idx(i + 2, j + 2, k + 2);
  const double tau_n = io.d_tau[0];
  const double tau_src = (STAGE == 1) ? tau_n : tau_n + P.dtau;
  const double tau_out = tau_n + P.dtau;
  double qn[NQ];  // the new conserved state (a harmless rest state on lanes past the edge)
#pragma unroll
  for (int n = 0; n < NQ; ++n) qn[n] = (n == 0) ? 1.0 : 0.0;

  if (valid) {
    R dq[NQ];
    cell_rhs<R, TH1, IFACE>(P, L, io, c, tau_src, dq, amax);

    // ---- c) Heun update in FP64 (Eqs. step1-finalStep)
#pragma unroll
    for (int n = 0; n < NQ; ++n) {
      const double qi = __ldg(io.q_in + n * fs + c);
      if (STAGE == 1)
        qn[n] = qi + to_f64<R>(dq[n] * pr<R>(P).dtau);  // q* = q^n + dtau C[q^n]
      else  // q^{n+1} = (q^n + q* + dtau C[q*]) / 2
        qn[n] = fma(0.5, io.q_base[n * fs + c] + qi, to_f64<R>(dq[n] * pr<R>(P).half_dtau));
    }
  }

  if (valid) {
    // ---- d) inversion at tau^{n+1}
    double e, P0;
    R uo[4];
    const double guess = to_f64<R>(ld<R>(io.e_in, c));
    st |= invert_fp64(P, tau_out, qn, guess, e, P0, uo, nit);

    // the new state in the stencil precision (the copy the next stage's stencil reads)
    R qr[NQ];
#pragma unroll
    for (int n = 0; n < NQ; ++n) qr[n] = from_f64<R>(qn[n]);
    const R eR = from_f64<R>(e), P0R = from_f64<R>(P0);

    // ---- e) regulator
    if (P.regulate) {
      const R go = P.milne ? from_f64<R>(tau_out * tau_out) : R(1);
      R pm[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
          pm[a][b] = qr[pix(a, b)];
          pm[b][a] = pm[a][b];
        }
      const R f = regulator_factor<R>(P, go, eR, P0R, uo, pm, qr[14]);
      if (f < R(0.999)) ++nreg;
      if (STAGE == 2 && io.reg_out) io.reg_out[c] = to_f32(f);
      if (f != R(1)) {
        const double fd = to_f64<R>(f);
#pragma unroll
        for (int n = 4; n < 14; ++n) {
          qn[n] *= fd;
          qr[n] *= f;
        }
      }
    }
#pragma unroll
    for (int n = 0; n < NQ; ++n)
      if (!isfinite(qr[n])) st |= ST_NONFINITE;

    // ---- f) stores
    store_with_ghosts<R>(P, L, io, i + 2, j + 2, k + 2, qn, qr, uo, eR, P0R);
  }
}

// The contiguous run [t0, t1) of the tile table that this block processes.  Tiles are ordered
// eta-fastest, so a block of a persistent grid walks up a column of tiles and the eta-neighbour
// planes read by its stencil are mostly still in its SM's L1.
__device__ __forceinline__ void tile_range(int ntiles, int& t0, int& t1) {
  const int per = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
  t0 = (int)blockIdx.x * per;
  t1 = min(ntiles, t0 + per);
}

// ---------------------------------------------------------------- per-launch statistics
// status bits OR-ed, the largest local speed (float bits, all non-negative), and the Newton /
// regulated / fallback counters: warp reductions, then one set of atomics per block.  Every
// thread of the block calls this once, after its last cell.
__device__ __forceinline__ void block_stats(unsigned* status, unsigned* max_speed_bits,
                                            unsigned long long* counters, unsigned st, float amax, unsigned nit,
                                            unsigned nreg, unsigned nfb) {
  __shared__ unsigned s_st[32], s_max[32], s_it[32], s_reg[32], s_fb[32];
  const unsigned full = 0xffffffffu;
  unsigned w_st = __reduce_or_sync(full, st);
  unsigned w_max = __reduce_max_sync(full, __float_as_uint(amax));
  unsigned w_it = __reduce_add_sync(full, nit);
  unsigned w_reg = __reduce_add_sync(full, nreg);
  unsigned w_fb = __reduce_add_sync(full, nfb);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int warp = tid >> 5, nwarps = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
  if ((tid & 31) == 0) {
    s_st[warp] = w_st; s_max[warp] = w_max; s_it[warp] = w_it; s_reg[warp] = w_reg; s_fb[warp] = w_fb;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned a = 0, b = 0, cI = 0, d = 0, fb = 0;
    for (int w = 0; w < nwarps; ++w) {
      a |= s_st[w]; b = max(b, s_max[w]); cI += s_it[w]; d += s_reg[w]; fb += s_fb[w];
    }
    if (a) atomicOr(status, a);
    if (max_speed_bits) atomicMax(max_speed_bits, b);
    if (cI) atomicAdd(counters + 0, (unsigned long long)cI);
    if (d) atomicAdd(counters + 1, (unsigned long long)d);
    if (fb) atomicAdd(counters + 2, (unsigned long long)fb);
  }
}

// ---------------------------------------------------------------- the stage kernel
// Persistent: every block walks its run of the tile table; a tile is one block-shaped patch of one
// event, so one launch per Runge-Kutta stage advances every event of the context.
template <typename R, int STAGE, bool TH1, bool IFACE>
__global__ void __launch_bounds__(256, 1)
    stage_kernel(const Params P, const StageIO<R> io, const Lattice* __restrict__ lats, const Tile* __restrict__ tiles,
                 int ntiles) {
  unsigned st = 0, nit = 0, nreg = 0;
  float amax = 0.f;
  int t0, t1;
  tile_range(ntiles, t0, t1);
  for (int t = t0; t < t1; ++t) {
    const Tile tl = tiles[t];
    const Lattice L = lats[tl.event];
    stage_cell<R, STAGE, TH1, IFACE>(P, L, io, tl.i0 + (int)threadIdx.x, tl.j0 + (int)threadIdx.y, tl.k0 + (int)threadIdx.z, st,
                         nit, nreg, amax);
  }

  block_stats(io.status, io.max_speed_bits, io.counters, st, amax, nit, nreg, 0u);
}

}  // namespace kt
