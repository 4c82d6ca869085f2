// kt_split.cuh -- the mixed-precision Runge-Kutta stage as two launches (or one fused launch).
//
// rhs_kernel<S>:    k_S = dtau C[q] in FP32 (a, b of the stage: stencil, fluxes, sources; Sec. 3.1,
//                   App. B).  No FP64 arithmetic, so it runs at the occupancy of the FP32 code.
// update_kernel<S>: the FP64 Heun accumulation, the root-find (learned start from the network's
//                   output of mlp_start_kernel, or the plain safeguarded Newton), the regulator and
//                   the stores (c-f).
// fused_kernel<S>:  both in one launch, k in shared memory.
// mlp_start_kernel: the network's output z for every cell at the start of the step (tensor cores).
//
// Heun (Eqs. step1-finalStep) in increment form:
//     q*      = q^n + k_1,            k_1 = dtau C[q^n]
//     q^{n+1} = (q^n + q* + k_2) / 2 = q^n + (k_1 + k_2) / 2,   k_2 = dtau C[q*],
// summed in FP64 onto q^n.  q* itself is never stored in FP64: the root-find of stage 1 forms the
// components it needs (T^{tau mu}, pi^{tau mu}, Pi) in FP64, the stage-2 stencil reads the FP32
// copy of q*, and the regulator's rescaling q* -> f q* of the pi components is carried in k_1 as
// f k_1 + (f - 1) q^n.  (Forming (k_1 + k_2)/2 in the stage-2 rhs kernel instead was measured
// slower: the read of k_1 at the end of that kernel costs more than it saves in the update.)
#pragma once
#include "kt_stage.cuh"
#include "kt_tma.cuh"

namespace kt {

struct UpdIO {
  double* q;                // q^n, FP64; stage 2 overwrites it with q^{n+1} (own cell only)
  const float* qf_n;        // FP32 copy of q^n (FP32 pi storage: components 4-14 are the state itself)
  const float* qsf;         // FP32 pi storage, stage 2: q* (its pi and Pi components are the state)
  float* k1;                // dtau C[q^n]; stage 1 rewrites its pi components with the regulated increment
  const float* k2;          // dtau C[q*] (stage 2)
  float* qr_out;            // FP32 copy of the new state: q* (stage 1) or q^{n+1} (stage 2), with ghosts
  float* u_out;
  float* e_out;
  float* p_out;
  const float* e_guess;     // the cell's previous energy density: the plain root-find's start
  const double* d_tau;      // tau^n
  unsigned* status;
  unsigned long long* counters;
  float* reg_out;           // stage 2: the regulation factor applied at each cell, or null
  const float* z_net;       // learned start: the network's output z per cell for the step (mlp_start_kernel)
};

// inversion inputs of q: T^{tau mu} (0-3), pi^{tau mu} (4-7), Pi (14)
__device__ __forceinline__ constexpr bool inversion_component(int n) { return n < 8 || n == 14; }

// Shared-memory staging of the stencil: per tile, the box of (bx+4) x (by+4) x (bz+4) FP32 values
// (the tile and its two-cell halo in x, y, eta) of kCompPerBox consecutive components is copied by
// one TMA load from the event's 4-d tensor map (x, y, eta, component) into one of two buffers, so
// that the copy of the next group overlaps the fluxes of the current one, with one block barrier
// per group.  Parts of a box beyond the padded lattice are zero-filled by TMA and read by no valid
// cell.  The buffers live in dynamic shared memory sized for the tile shape (rhs_smem_bytes).
constexpr int kBoxMax = 2176;               // floats per component box: >= 36 * 12 * 5, a multiple of 32
constexpr int kCompPerBox = 3;              // components per TMA load (15 = 5 groups)
constexpr int kGroups = (NQ + kCompPerBox - 1) / kCompPerBox;
constexpr unsigned kWaitPolls = 1u << 20;   // mbarrier polls before a wait gives up (far beyond any copy)
__host__ __device__ constexpr int rhs_buffer_floats(int tx, int ty, int tz) {  // 128-byte multiple
  return (kCompPerBox * (tx + 4) * (ty + 4) * (tz + 4) + 31) & ~31;
}
__host__ __device__ constexpr int rhs_smem_bytes(int tx, int ty, int tz) {  // two buffers + alignment slack
  return 4 * (2 * rhs_buffer_floats(tx, ty, tz) + 32);
}

// Register caps: 96 (rhs) lets 20 warps of 128-thread tiles share an SM; 72 (stage-1 update) 28
// warps; 96 for the stage-2 update, which holds all 15 FP64 components.  Each measured faster than
// the compiler's unconstrained choice; for the update kernels, caps of 64-80 (stage 1) and 72-96
// (stage 2) all measure within 0.5% of each other (latency-bound: more warps, more spills).
template <int STAGE, bool TH1, bool IFACE>
__global__ void __maxnreg__(96)
    rhs_kernel(const Params P, const StageIO<float> io, float* __restrict__ k_out, const Lattice* __restrict__ lats,
               const Tile* __restrict__ tiles, int ntiles, const CUtensorMap* __restrict__ tmaps) {
  extern __shared__ __align__(128) float s_raw[];
  __shared__ alignas(8) uint64_t s_bar[2];
  float* const s_q = s_raw + ((32u - ((smem_u32(s_raw) >> 2) & 31u)) & 31u);  // TMA wants 128-byte buffers
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int bx = blockDim.x + 4, by = blockDim.y + 4, bz = blockDim.z + 4;
  const int vol = bx * by * bz;                  // floats per component in a buffer
  const unsigned box_bytes = 4u * kCompPerBox * vol;
  const int bfl = rhs_buffer_floats(blockDim.x, blockDim.y, blockDim.z);
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();

  float amax = 0.f;
  bool bad = false;
  unsigned issued = 0, done = 0;  // TMA copies issued and waited for (the same in every thread)
  const double tau_n = io.d_tau[0];
  const CellGeom<float> G = cell_geom<float>(P, (STAGE == 1) ? tau_n : tau_n + P.dtau);
  const float th = pr<float>(P).theta;
  const int sy = bx, sz = bx * by;
  const int own = ((int)threadIdx.z + 2) * sz + ((int)threadIdx.y + 2) * sy + (int)threadIdx.x + 2;
  auto stage_group = [&](const CUtensorMap* map, const Tile& tl, int g) {  // thread 0 only
    const unsigned b = issued & 1u;
    fence_proxy_async_smem();  // earlier reads of this buffer before the async-proxy write
    mbar_arrive_expect_tx(&s_bar[b], box_bytes);
    tma_load_4d(s_q + b * bfl, map, tl.i0, tl.j0, tl.k0, kCompPerBox * g, &s_bar[b]);
  };

  int t0, t1;
  tile_range(ntiles, t0, t1);
  for (int t = t0; t < t1; ++t) {
    const Tile tl = tiles[t];
    const Lattice L = lats[tl.event];
    const CUtensorMap* map = tmaps + tl.event;
    if (__syncthreads_or(bad)) { bad = true; break; }  // every thread is done with both buffers
    if (tid == 0) {
      fence_tensormap_acquire(map);
      stage_group(map, tl, 0);
    }
    ++issued;

    const int i = tl.i0 + (int)threadIdx.x, j = tl.j0 + (int)threadIdx.y, k = tl.k0 + (int)threadIdx.z;
    const bool valid = (i < L.nx) && (j < L.ny) && (k < L.nz);
    const long long c = valid ? L.idx(i + 2, j + 2, k + 2) : 0;
    float dq[NQ], uc[4], du[4][4], dv = 0.f;
    Faces<float> Fx, Fy, Fz;
    if (valid) {  // the sources first: du and dv are dead before the component loop (fewer spills)
      cell_faces<float, TH1, IFACE>(P, L, io, c, u_global(L, io, c), G, dq, uc, du, dv, amax, Fx, Fy, Fz);
      cell_sources<float>(P, L, io, c, G, uc, du, dv, dq);
    }

    const FacesXY Wxy = faces_xy(Fx, Fy);  // theta = 1: the x and y fluxes in paired instructions
#pragma unroll  // unrolled: the component index, the rows it feeds and every branch become constants
    for (int g = 0; g < kGroups; ++g) {
      if (g + 1 < kGroups) {
        if (__syncthreads_or(bad)) { bad = true; break; }  // the other buffer is free again
        if (tid == 0) stage_group(map, tl, g + 1);
        ++issued;
      }
      const unsigned b = done & 1u;
      if (!mbar_wait(&s_bar[b], (done >> 1) & 1u, kWaitPolls)) { bad = true; continue; }
      ++done;
      if (valid) {
#pragma unroll
        for (int m = 0; m < kCompPerBox; ++m)
          if (kCompPerBox * g + m < NQ) {
            if constexpr (TH1)
              component_rhs_xy(P, kCompPerBox * g + m, s_q + b * bfl + m * vol + own, sy, sz, Wxy, Fx, Fy, Fz, dq);
            else
              component_rhs<float, true, TH1>(P, kCompPerBox * g + m, s_q + b * bfl + m * vol + own, 1, sy, sz, th,
                                              Fx, Fy, Fz, dq);
          }
      }
    }
    if (valid && !bad) {  // (a timed-out block leaves at the next tile's barrier)
      const float dt = pr<float>(P).dtau;
#pragma unroll
      for (int n = 0; n < NQ; ++n) k_out[n * L.fstride + c] = dq[n] * dt;
    }
  }
  if (bad) {  // a copy did not complete in time: let the ones in flight land before the block exits
    for (; done < issued; ++done) mbar_wait(&s_bar[done & 1u], (done >> 1) & 1u, kWaitPolls);
  }
  block_stats(io.status, io.max_speed_bits, io.counters, bad ? ST_TIMEOUT : 0u, amax, 0u, 0u, 0u);
}

// ------------------------------------------------------------- d) the root-find (Sec. 2.4)
// Learned start: from e_start at most two Newton steps; the root is accepted as soon as
// |f(e)| <= 1e-10 E, i.e. |g| <= 1e-10 E A; otherwise the plain root-find continues from the
// last iterate and the cell counts as a fallback.  The test costs no FP64 instruction: the
// threshold 0.99e-10 E A is formed in single precision from E and A truncated, and |g| is
// compared with it on the upper 32 bits of both doubles (strictly below).  The 1% margin covers
// the single-precision rounding of the threshold and the mixed records' P0 (g is evaluated with
// P0 within ~2e-13 E A of the FP64 cubic's inside the table), so an accepted root satisfies
// the exact test.
__device__ __forceinline__ unsigned abs_hi(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }
// upper 32 bits of the double equal to the positive normal float t (0 for a smaller or non-finite t)
__device__ __forceinline__ unsigned thr_hi(float t) {
  const unsigned b = __float_as_uint(t);
  return (b >= 0x00800000u && b < 0x7f800000u) ? (b >> 3) + (896u << 20) : 0u;
}
__device__ __forceinline__ unsigned rootfind_learned(const Params& P, const InvIn& v, double EPi, double e_start,
                                                     double& e, double& P0, unsigned& iters, unsigned& fallbacks) {
  const double lo = (P.e_min > 0.0) ? P.e_min : 1e-300;
  // (E >= 2^120, beyond where the truncated E and A are valid single-precision values: no
  // acceptance, the plain root-find decides)
  const float tolf = (obits(v.E) < 0x4770000000000000LL) ? 0.99e-10f * v.Ef : 0.f;
  e = clamp_pos(e_start, lo, v.E);
#pragma unroll 1
  for (int kk = 0; kk < 3; ++kk) {
    const Resid r = residual<true>(P, e, v.E, EPi, v.M2, v.M2f);
    if (abs_hi(r.g) < thr_hi(tolf * r.Af)) {
      P0 = r.p0;
      return 0u;
    }
    if (kk == 2) break;
    e = clamp_pos(newton_step(e, r), lo, v.E);
    ++iters;
  }
  ++fallbacks;
  return rootfind_plain(P, v.E, EPi, v.M2, v.M2f, e, e, P0, iters);
}

// (E, M^i, Pi) -> (e, P0, u^mu) at tau^{n+1} for the mixed path (Eqs. eInferred-uiInferred).  With
// the conformal EOS and no bulk pressure the closed form e = sqrt(4E^2 - 3M^2) - E is used.
// M^2 < E^2 is decided in single precision, with a margin, where E and M^2 lie well inside its
// range (M^2 < 0.998 E^2 in the truncated values makes it certain), else by the FP64 product.
template <bool LEARNED>
__device__ __forceinline__ unsigned invert_split(const Params& P, const InvIn& v, double start, double& e,
                                                 double& P0, float (&uo)[4], unsigned& iters, unsigned& fallbacks) {
  const double E = v.E, M2 = v.M2, Pi = v.Pi;
  const long long bE = obits(E), bM2 = obits(M2);
  bool ok = bE > 0 && bE < 0x7ff0000000000000LL;  // E > 0 finite
  if (ok && !(bE > 0x3c30000000000000LL && bE < 0x43b0000000000000LL && bM2 < 0x4770000000000000LL &&
              v.M2f < 0.998f * v.Ef * v.Ef))  // 2^-60 < E < 2^60, M^2 < 2^120
    ok = bM2 < obits(E * E);
  unsigned st = 0;
  if (!ok) {
    st = ST_INVERSION;
    e = (P.e_min > 0.0) ? P.e_min : 1e-30;
    P0 = e * (1.0 / 3.0);
  } else if (!P.eos_table) {
    if (P.bulk_on && Pi != 0.0) {
      st = ST_INVERSION;  // bulk pressure needs a non-conformal EOS
      e = E;
    } else {
      const double M = sqrt(M2);  // cancellation-free form of sqrt(4E^2 - 3M^2) - E
      e = 3.0 * (E - M) * (E + M) / (sqrt(fma(4.0 * E, E, -3.0 * M2)) + E);
    }
    P0 = e * (1.0 / 3.0);
  } else if (LEARNED) {
    st = rootfind_learned(P, v, E + Pi, start, e, P0, iters, fallbacks);
  } else {
    st = rootfind_plain(P, E, E + Pi, M2, v.M2f, start, e, P0, iters);
  }
  if (st) {
    uo[0] = 1.f;
    uo[1] = uo[2] = uo[3] = 0.f;
  } else {
    // u^tau = sqrt((E + P)/(e + P)), u^i = M^i / ((e + P) u^tau), P = P0 + Pi, in single precision
    const float Pt = d2f_bits(P0) + d2f_bits(Pi);
    const float ePt = d2f_bits(e) + Pt, EPt = d2f_bits(E) + Pt;
    const float ut = sqrtf(__fdividef(EPt, ePt));
    const float w = __fdividef(1.f, ePt * ut);
    uo[0] = ut;
    uo[1] = d2f_bits(v.Mx) * w;
    uo[2] = d2f_bits(v.My) * w;
    uo[3] = d2f_bits(v.Mn) * w;
  }
  if (!isfinite(uo[0]) || !isfinite(uo[1]) || !isfinite(uo[2]) || !isfinite(uo[3]) ||
      !((obits(e) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL))
    st |= ST_NONFINITE;
  return st;
}

// Where the update of one cell reads its inputs: straight from the field arrays (UpdInGlobal), or
// from the tile's box staged in shared memory by TMA (UpdInShared, below).  q(n): q^n in FP64;
// k1(n), k2(n): the stage increments; qfn(n): the FP32 copy of q^n (stage 1); qs(n): the FP32 q*
// (FP32 pi storage, stage 2).
struct UpdInGlobal {
  const UpdIO& io;
  long long fs, c;
  __device__ __forceinline__ double q(int n) const { return __ldg(io.q + n * fs + c); }
  __device__ __forceinline__ float k1(int n) const { return __ldg(io.k1 + n * fs + c); }
  __device__ __forceinline__ float k2(int n) const { return __ldg(io.k2 + n * fs + c); }
  __device__ __forceinline__ float qfn(int n) const { return __ldg(io.qf_n + n * fs + c); }
  __device__ __forceinline__ float qs(int n) const { return __ldg(io.qsf + n * fs + c); }
};

// the increment added to q^n in FP64: k_1 (stage 1) or (k_1 + k_2)/2 (stage 2)
template <int STAGE, typename In>
__device__ __forceinline__ float increment(const In& in, int n) {
  if constexpr (STAGE == 1) return in.k1(n);
  else return 0.5f * (in.k1(n) + in.k2(n));
}

// FP32 pi storage (KT_STORE_PI_FP32): pi^{mu nu} and Pi are the FP32 values of the stencil copy,
// Heun-summed in FP32; only T^{tau mu} (components 0-3) is kept and summed in FP64.  The new pi, Pi
// of one cell: q* = q^n + k_1 (stage 1) or q^{n+1} = (q^n + q* + k_2)/2 (stage 2), Eqs. (step1)-
// (finalStep), with q* the regulated first-stage state.
template <int STAGE, typename In>
__device__ __forceinline__ float pi32_state(const In& in, int n) {
  if constexpr (STAGE == 1) return in.qfn(n) + in.k1(n);
  else return 0.5f * (in.qfn(n) + in.qs(n) + in.k2(n));
}

// One cell; all lanes of the warp call it together (the learned start is warp-wide).  STORE_K1
// (stage 1 of the fused stage kernel, whose k_1 exists only in shared memory): write all of k_1
// to the field array for the second stage, its pi components carrying the regulator's rescaling.
template <int STAGE, bool LEARNED, bool PI32, typename In, bool STORE_K1 = false>
__device__ __forceinline__ void update_cell(const Params& P, const Lattice& L, const UpdIO& io, const In& in, int i,
                                            int j, int k, double tau_out, unsigned& st,
                                            unsigned& nit, unsigned& nreg, unsigned& nfb) {
  const bool valid = (i < L.nx) && (j < L.ny) && (k < L.nz);
  const long long fs = L.fstride;
  const long long c = L.idx(i + 2, j + 2, k + 2);
  double qn[NQ];  // FP64 new state; components outside the inversion set are formed after it
  float qp[NQ];   // FP32 pi storage: the new pi, Pi (components 4-14)
#pragma unroll
  for (int n = 0; n < NQ; ++n) qn[n] = (n == 0) ? 1.0 : 0.0;  // a harmless rest state past the edge
  // Stage 1 with FP64 pi storage stores no FP64 state: the inversion's E = (T^tt - pi^tt) + the
  // single-precision difference of their increments in k_1 (likewise M^i), two FP64 additions
  // per pair instead of three; otherwise E, M^i are differences of the new FP64 components.
  constexpr bool kDiff = (STAGE == 1) && !PI32;
  double E = 1.0, Mx = 0.0, My = 0.0, Mn = 0.0, Pi = 0.0;
  if (valid) {
    if constexpr (kDiff) {
      E = (in.q(0) - in.q(4)) + to_f64<float>(in.k1(0) - in.k1(4));
      Mx = (in.q(1) - in.q(5)) + to_f64<float>(in.k1(1) - in.k1(5));
      My = (in.q(2) - in.q(6)) + to_f64<float>(in.k1(2) - in.k1(6));
      Mn = (in.q(3) - in.q(7)) + to_f64<float>(in.k1(3) - in.k1(7));
      Pi = in.q(14) + to_f64<float>(in.k1(14));
    } else {
#pragma unroll
      for (int n = 0; n < NQ; ++n) {
        if (PI32 && n >= 4) {
          qp[n] = pi32_state<STAGE>(in, n);
          if (inversion_component(n)) qn[n] = to_f64<float>(qp[n]);  // exact widening for E, M^i, Pi
        } else if (inversion_component(n)) {
          qn[n] = in.q(n) + to_f64<float>(increment<STAGE>(in, n));
        }
      }
      E = qn[0] - qn[4];
      Mx = qn[1] - qn[5];
      My = qn[2] - qn[6];
      Mn = qn[3] - qn[7];
      Pi = qn[14];
    }
  }

  const double gnn = P.milne ? tau_out * tau_out : 1.0;
  const InvIn v = inv_in(gnn, E, Mx, My, Mn, Pi);
  double start;
  if constexpr (LEARNED) {
    start = learned_start(v, valid ? __ldg(io.z_net + c) : 0.f);
  } else {
    start = valid ? to_f64<float>(__ldg(io.e_guess + c)) : 1.0;
  }

  if (!valid) return;
  double e, P0;
  float uo[4];
  st |= invert_split<LEARNED>(P, v, start, e, P0, uo, nit, nfb);

  // the FP32 copy read by the next stencil (and the remaining FP64 components in stage 2)
  // Stage 2 forms pi components 8-13 as f q^n + f dq in one FP64 multiply-add once the
  // regulation factor f is known (measured faster than the separate sum and product).
  constexpr bool kFusePi = (STAGE == 2) && !PI32;
  float qr[NQ];
  double q8[6];  // q^n and the increment of pi components 8-13 (kFusePi)
  float inc8[6];
  bool scaled = false;
  if constexpr (PI32) {
#pragma unroll
    for (int n = 0; n < NQ; ++n) {
      if (n >= 4) qr[n] = qp[n];
      else if (STAGE == 1) qr[n] = in.qfn(n) + in.k1(n);
      else qr[n] = from_f64<float>(qn[n]);
    }
  } else if constexpr (STAGE == 1) {
#pragma unroll
    for (int n = 0; n < NQ; ++n) qr[n] = in.qfn(n) + in.k1(n);
  } else if constexpr (kFusePi) {  // the pi components outside the inversion set are read once, here
#pragma unroll
    for (int n = 0; n < NQ; ++n) {
      if (!inversion_component(n)) {
        q8[n - 8] = in.q(n);
        inc8[n - 8] = increment<STAGE>(in, n);
        qr[n] = from_f64<float>(q8[n - 8]) + inc8[n - 8];
      } else {
        qr[n] = from_f64<float>(qn[n]);
      }
    }
  } else {
#pragma unroll
    for (int n = 0; n < NQ; ++n) {
      if (!inversion_component(n)) qn[n] = in.q(n) + to_f64<float>(increment<STAGE>(in, n));
      qr[n] = from_f64<float>(qn[n]);
    }
  }
  const float eR = from_f64<float>(e), P0R = from_f64<float>(P0);

  // e) regulator (Eq. regPimunu), after the root-find, on pi only
  bool k1_pi_written = false;  // STORE_K1: the pi components of k_1 were written rescaled
  if (P.regulate) {
    const float go = P.milne ? from_f64<float>(tau_out * tau_out) : 1.f;
    float pm[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a; b < 4; ++b) {
        pm[a][b] = qr[pix(a, b)];
        pm[b][a] = pm[a][b];
      }
    const float f = regulator_factor<float>(P, go, eR, P0R, uo, pm, qr[14]);
    if (f < 0.999f) ++nreg;
    if (STAGE == 2 && io.reg_out) io.reg_out[c] = f;
    if (f != 1.f) {
      if constexpr (PI32) {  // the FP32 state itself is rescaled (stage 2 reads q* from it)
#pragma unroll
        for (int n = 4; n < 14; ++n) qr[n] *= f;
      } else if constexpr (STAGE == 1) {
#pragma unroll
        for (int n = 4; n < 14; ++n) {  // f q* = q^n + (f k_1 + (f - 1) q^n)
          io.k1[n * fs + c] = fmaf(f, in.k1(n), (f - 1.f) * in.qfn(n));
          qr[n] *= f;
        }
        k1_pi_written = true;
      } else {  // rescale the FP64 state in registers (re-reading its inputs would miss L2)
        const double fd = to_f64<float>(f);
#pragma unroll
        for (int n = 4; n < 14; ++n) {
          if (!kFusePi || n < 8) qn[n] *= fd;
          else qn[n] = fma(fd, q8[n - 8], to_f64<float>(f * inc8[n - 8]));
          qr[n] *= f;
        }
        scaled = true;
      }
    }
  }
  if constexpr (kFusePi) {
    if (!scaled) {
#pragma unroll
      for (int n = 8; n < 14; ++n) qn[n] = q8[n - 8] + to_f64<float>(inc8[n - 8]);
    }
  }
  if constexpr (STORE_K1 && STAGE == 1 && !PI32) {
#pragma unroll
    for (int n = 0; n < NQ; ++n)
      if (n < 4 || n > 13 || !k1_pi_written) io.k1[n * fs + c] = in.k1(n);
  }
#pragma unroll
  for (int n = 0; n < NQ; ++n)
    if (!isfinite(qr[n])) st |= ST_NONFINITE;

  // f) stores: q^{n+1} in FP64 at the cell (no kernel reads its ghosts), the FP32 copy, u, e, P
  //    at the cell and its ghosts
  if constexpr (STAGE == 2) {
#pragma unroll
    for (int n = 0; n < NQ; ++n)
      if (!PI32 || n < 4) io.q[n * fs + c] = qn[n];
  }
  for_cell_and_ghosts(P, L, i + 2, j + 2, k + 2, [&](long long t) {
#pragma unroll
    for (int n = 0; n < NQ; ++n) io.qr_out[n * fs + t] = qr[n];
#pragma unroll
    for (int m = 0; m < 4; ++m) io.u_out[m * fs + t] = uo[m];
    io.e_out[t] = eR;
    io.p_out[t] = P0R;
  });
}

template <int STAGE, bool LEARNED, bool PI32>
__global__ void __maxnreg__(STAGE == 1 ? 72 : 96)
    update_kernel(const Params P, const UpdIO io, const Lattice* __restrict__ lats, const Tile* __restrict__ tiles,
                  int ntiles) {
  unsigned st = 0, nit = 0, nreg = 0, nfb = 0;
  const double tau_out = io.d_tau[0] + P.dtau;
  int t0, t1;
  tile_range(ntiles, t0, t1);
  for (int t = t0; t < t1; ++t) {
    const Tile tl = tiles[t];
    const Lattice L = lats[tl.event];
    const int i = tl.i0 + (int)threadIdx.x, j = tl.j0 + (int)threadIdx.y, k = tl.k0 + (int)threadIdx.z;
    const UpdInGlobal in{io, L.fstride, L.idx(i + 2, j + 2, k + 2)};
    update_cell<STAGE, LEARNED, PI32>(P, L, io, in, i, j, k, tau_out, st, nit, nreg, nfb);
  }
  block_stats(io.status, nullptr, io.counters, st, 0.f, nit, nreg, nfb);
}

// ---------------------------------------------------------------- the network, once per step
// The learned start's network output z for every element of the field arrays (cells, their
// ghosts and the padding between events) from the FP32 copy of the state q^n at tau^n, before the
// first stage: one warp per 32 consecutive elements (coalesced loads of the 9 components the
// features read), the warp-wide tensor-core inference where one of its elements has r^2 above
// kMlpGateR2 (else z = 0).  Both stages of the step apply this z to their own E, M^2 and Pi, which
// differ from q^n by O(dtau).  Run in a launch of its own, at full occupancy, the inference's
// latency hides behind other warps; inside the register-capped update it could not.
__global__ void __launch_bounds__(256) mlp_start_kernel(const float* __restrict__ qf, long long fs,
                                                        const double* __restrict__ d_tau, int milne,
                                                        const uint32_t* __restrict__ packed,
                                                        float* __restrict__ z_net) {
  __shared__ alignas(16) uint32_t sw[PK_WORDS];
  mlp_load_shared(sw, packed);
  __syncthreads();
  const float tau = d2f_trunc(d_tau[0]);
  const float gnn = milne ? tau * tau : 1.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < fs; base += stride) {  // block-uniform
    const long long t = base + threadIdx.x;
    const bool in = t < fs;
    float E = 1.f, Mx = 0.f, My = 0.f, Mn = 0.f, Pi = 0.f;  // a rest state past the end
    if (in) {
      E = __ldg(qf + t) - __ldg(qf + 4 * fs + t);
      Mx = __ldg(qf + fs + t) - __ldg(qf + 5 * fs + t);
      My = __ldg(qf + 2 * fs + t) - __ldg(qf + 6 * fs + t);
      Mn = __ldg(qf + 3 * fs + t) - __ldg(qf + 7 * fs + t);
      Pi = __ldg(qf + 14 * fs + t);
    }
    float x[MLP_IN], ecE;
    mlp_features(fmaxf(E, 1e-30f), fmaf(Mx, Mx, fmaf(My, My, gnn * Mn * Mn)), Pi, x, ecE);
    const float z = __any_sync(0xffffffffu, x[1] > kMlpGateR2) ? mlp_warp_infer(sw, x) : 0.f;  // all lanes
    if (in) z_net[t] = z;
  }
}

// ---------------------------------------------------------------- staged update (TMA)
// The inputs of a tile's update (FP64 pi storage) are copied into shared memory by a few TMA bulk
// loads instead of one global load per thread and component, so that the loads of a tile are all
// in flight at once without holding registers: stage 1 q^n components 0-7 and 14 (FP64), k_1 and
// the FP32 copy of q^n (15 each); stage 2 q^n (15, FP64), k_1 and k_2.  A box spans the tile's
// cells in y and eta and bx + 4 cells in x, from the tile's padded x (a multiple of 32, so that
// every copy starts on a 16-byte boundary); a thread's own cell sits at x offset 2.  Blocks of a
// persistent grid double-buffer: the next tile's copies land while the current tile computes.
constexpr int kUpdQSlots = 16;  // FP64 component slots: two boxes of 8 (stage 1 uses 9)
constexpr int kUpdMaps = 5;     // tensor maps per event: q (8 deep), q (1 deep), k_1, k_2, FP32 copy of q
__host__ __device__ constexpr int upd_box_cells(int tx, int ty, int tz) { return (tx + 4) * ty * tz; }
__host__ __device__ constexpr int upd_align128(int b) { return (b + 127) & ~127; }
__host__ __device__ constexpr int upd_buffer_bytes(int tx, int ty, int tz) {
  return upd_align128(kUpdQSlots * 8 * upd_box_cells(tx, ty, tz)) + 2 * upd_align128(NQ * 4 * upd_box_cells(tx, ty, tz));
}
__host__ __device__ constexpr int upd_smem_bytes(int tx, int ty, int tz, int nbuf) {
  return nbuf * upd_buffer_bytes(tx, ty, tz) + 128;  // + alignment slack
}

template <int STAGE>
struct UpdInShared {
  const double* sq;  // q^n: slot n (stage 1: component 14 in slot 8), bc cells per slot
  const float* sa;   // k_1, component n at n * bc
  const float* sb;   // stage 1: the FP32 copy of q^n; stage 2: k_2
  int bc, own;
  __device__ __forceinline__ double q(int n) const { return sq[((STAGE == 1 && n == 14) ? 8 : n) * bc + own]; }
  __device__ __forceinline__ float k1(int n) const { return sa[n * bc + own]; }
  __device__ __forceinline__ float k2(int n) const { return sb[n * bc + own]; }
  __device__ __forceinline__ float qfn(int n) const { return sb[n * bc + own]; }
  __device__ __forceinline__ float qs(int) const { return 0.f; }  // (FP32 pi storage is not staged)
};

template <int STAGE, bool LEARNED>
__global__ void __maxnreg__(STAGE == 1 ? 72 : 96)
    update_staged_kernel(const Params P, const UpdIO io, const Lattice* __restrict__ lats,
                         const Tile* __restrict__ tiles, int ntiles, const CUtensorMap* __restrict__ umaps, int nbuf) {
  extern __shared__ __align__(128) unsigned char u_raw[];
  __shared__ alignas(8) uint64_t s_bar[2];
  unsigned char* const sbase = u_raw + ((128u - (smem_u32(u_raw) & 127u)) & 127u);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int bc = (blockDim.x + 4) * blockDim.y * blockDim.z;
  const int qbytes = upd_align128(kUpdQSlots * 8 * bc), kbytes = upd_align128(NQ * 4 * bc);
  const int bufbytes = qbytes + 2 * kbytes;
  const unsigned q8_bytes = 64u * bc, q1_bytes = 8u * bc, k_bytes = 4u * NQ * bc;
  const unsigned tile_bytes = (STAGE == 1) ? (q8_bytes + q1_bytes + 2 * k_bytes) : (2 * q8_bytes + 2 * k_bytes);
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();

  unsigned st = 0, nit = 0, nreg = 0, nfb = 0;
  bool bad = false;
  unsigned issued = 0, done = 0;  // tiles whose copies were issued / waited for (the same in every thread)
  const double tau_out = io.d_tau[0] + P.dtau;
  int t0, t1;
  tile_range(ntiles, t0, t1);
  auto issue = [&](int t, unsigned slot) {  // thread 0 only: the four (stage 2) or five copies of tile t
    const Tile tl = tiles[t];
    const CUtensorMap* m = umaps + kUpdMaps * tl.event;
    unsigned char* buf = sbase + slot * bufbytes;
    uint64_t* bar = &s_bar[slot];
    for (int w = 0; w < kUpdMaps; ++w) fence_tensormap_acquire(m + w);
    fence_proxy_async_smem();  // earlier reads of this buffer before the async-proxy writes
    mbar_arrive_expect_tx(bar, tile_bytes);
    const int x = tl.i0, y = tl.j0 + 2, z = tl.k0 + 2;
    tma_load_4d(buf, m + 0, x, y, z, 0, bar);  // q^n components 0-7
    if constexpr (STAGE == 1) tma_load_4d(buf + q8_bytes, m + 1, x, y, z, 14, bar);  // component 14
    else tma_load_4d(buf + q8_bytes, m + 0, x, y, z, 8, bar);  // components 8-14 (15: zero fill)
    tma_load_4d(buf + qbytes, m + 2, x, y, z, 0, bar);  // k_1
    tma_load_4d(buf + qbytes + kbytes, m + ((STAGE == 1) ? 4 : 3), x, y, z, 0, bar);  // q^n copy / k_2
  };

  if (t0 < t1) {
    if (tid == 0) issue(t0, 0u);
    issued = 1;
  }
  for (int t = t0; t < t1; ++t) {
    if (nbuf == 2 && t + 1 < t1) {  // the other buffer was last read by the previous tile
      if (__syncthreads_or(bad)) { bad = true; break; }
      if (tid == 0) issue(t + 1, issued & 1u);
      ++issued;
    }
    const unsigned slot = (nbuf == 2) ? (done & 1u) : 0u;
    const unsigned parity = (nbuf == 2) ? ((done >> 1) & 1u) : (done & 1u);
    const bool ok = mbar_wait(&s_bar[slot], parity, kWaitPolls);
    if (ok) ++done;
    if (__syncthreads_or(!ok)) { bad = true; break; }  // every thread computes, or none
    const Tile tl = tiles[t];
    const Lattice L = lats[tl.event];
    const unsigned char* buf = sbase + slot * bufbytes;
    const int own = ((int)threadIdx.z * (int)blockDim.y + (int)threadIdx.y) * ((int)blockDim.x + 4) + (int)threadIdx.x + 2;
    const UpdInShared<STAGE> in{(const double*)buf, (const float*)(buf + qbytes), (const float*)(buf + qbytes + kbytes),
                                bc, own};
    update_cell<STAGE, LEARNED, false>(P, L, io, in, tl.i0 + (int)threadIdx.x, tl.j0 + (int)threadIdx.y,
                                       tl.k0 + (int)threadIdx.z, tau_out, st, nit, nreg, nfb);
    if (nbuf == 1 && t + 1 < t1) {  // single buffer: refill it once every thread is done with it
      if (__syncthreads_or(bad)) { bad = true; break; }
      if (tid == 0) issue(t + 1, 0u);
      ++issued;
    }
  }
  if (bad) {  // a copy did not complete in time: let the ones in flight land before the block exits
    for (; done < issued; ++done)
      mbar_wait(&s_bar[(nbuf == 2) ? (done & 1u) : 0u], (nbuf == 2) ? ((done >> 1) & 1u) : (done & 1u), kWaitPolls);
  }
  block_stats(io.status, nullptr, io.counters, st | (bad ? ST_TIMEOUT : 0u), 0.f, nit, nreg, nfb);
}

// ---------------------------------------------------------------- fused stage (one launch per stage)
// The right-hand side and the update of a tile in one kernel: the FP32 stencil of rhs_kernel gives
// k = dtau C[q] in registers, which goes to shared memory (the staging buffer the last-but-one
// component group used, free by then) instead of a field array, and the update of update_kernel
// reads it from there.  Each stage thus skips the write and read of its k (120 B per cell), and
// blocks of an SM in different phases keep the FP32 pipes (stencil) and the FP64 pipe (Heun sums,
// root-find) busy at the same time.  Stage 1 still writes k_1 for the second stage's Heun sum.
template <int STAGE>
struct UpdInFused {
  const UpdIO& io;
  long long fs, c;
  const float* sk;  // this stage's k: component n at sk[n * kst]
  int kst;
  __device__ __forceinline__ double q(int n) const { return __ldg(io.q + n * fs + c); }
  __device__ __forceinline__ float k1(int n) const {
    if constexpr (STAGE == 1) return sk[n * kst];
    else return __ldg(io.k1 + n * fs + c);
  }
  __device__ __forceinline__ float k2(int n) const { return sk[n * kst]; }
  __device__ __forceinline__ float qfn(int n) const { return __ldg(io.qf_n + n * fs + c); }
  __device__ __forceinline__ float qs(int) const { return 0.f; }  // (FP32 pi storage is not fused)
};

// 128 registers (16 warps of 128-thread tiles per SM): with the rhs kernel's 96 the two phases
// spilled 500 bytes per thread and the launch ran 10% slower.
template <int STAGE, bool TH1, bool IFACE, bool LEARNED>
__global__ void __maxnreg__(128)
    fused_kernel(const Params P, const StageIO<float> io, const UpdIO uio, const Lattice* __restrict__ lats,
                 const Tile* __restrict__ tiles, int ntiles, const CUtensorMap* __restrict__ tmaps) {
  extern __shared__ __align__(128) float s_raw[];
  __shared__ alignas(8) uint64_t s_bar[2];
  float* const s_q = s_raw + ((32u - ((smem_u32(s_raw) >> 2) & 31u)) & 31u);  // TMA wants 128-byte buffers
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int bx = blockDim.x + 4, by = blockDim.y + 4, bz = blockDim.z + 4;
  const int vol = bx * by * bz;                  // floats per component in a buffer
  const unsigned box_bytes = 4u * kCompPerBox * vol;
  const int bfl = rhs_buffer_floats(blockDim.x, blockDim.y, blockDim.z);
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();

  float amax = 0.f;
  bool bad = false;
  unsigned issued = 0, done = 0;  // TMA copies issued and waited for (the same in every thread)
  unsigned st = 0, nit = 0, nreg = 0, nfb = 0;
  const double tau_n = io.d_tau[0];
  const double tau_out = tau_n + P.dtau;
  const CellGeom<float> G = cell_geom<float>(P, (STAGE == 1) ? tau_n : tau_out);
  const float th = pr<float>(P).theta;
  const int sy = bx, sz = bx * by;
  const int own = ((int)threadIdx.z + 2) * sz + ((int)threadIdx.y + 2) * sy + (int)threadIdx.x + 2;
  auto stage_group = [&](const CUtensorMap* map, const Tile& tl, int g) {  // thread 0 only
    const unsigned b = issued & 1u;
    fence_proxy_async_smem();  // earlier accesses of this buffer before the async-proxy write
    mbar_arrive_expect_tx(&s_bar[b], box_bytes);
    tma_load_4d(s_q + b * bfl, map, tl.i0, tl.j0, tl.k0, kCompPerBox * g, &s_bar[b]);
  };

  int t0, t1;
  tile_range(ntiles, t0, t1);
  for (int t = t0; t < t1; ++t) {
    const Tile tl = tiles[t];
    const Lattice L = lats[tl.event];
    const CUtensorMap* map = tmaps + tl.event;
    if (__syncthreads_or(bad)) { bad = true; break; }  // every thread is done with both buffers
    if (tid == 0) {
      fence_tensormap_acquire(map);
      stage_group(map, tl, 0);
    }
    ++issued;

    const int i = tl.i0 + (int)threadIdx.x, j = tl.j0 + (int)threadIdx.y, k = tl.k0 + (int)threadIdx.z;
    const bool valid = (i < L.nx) && (j < L.ny) && (k < L.nz);
    const long long c = valid ? L.idx(i + 2, j + 2, k + 2) : 0;
    // ---- the right-hand side (as rhs_kernel)
    float dq[NQ], uc[4], du[4][4], dv = 0.f;
    Faces<float> Fx, Fy, Fz;
    if (valid) {
      cell_faces<float, TH1, IFACE>(P, L, io, c, u_global(L, io, c), G, dq, uc, du, dv, amax, Fx, Fy, Fz);
      cell_sources<float>(P, L, io, c, G, uc, du, dv, dq);
    }
    const FacesXY Wxy = faces_xy(Fx, Fy);
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
      if (g + 1 < kGroups) {
        if (__syncthreads_or(bad)) { bad = true; break; }
        if (tid == 0) stage_group(map, tl, g + 1);
        ++issued;
      }
      const unsigned b = done & 1u;
      if (!mbar_wait(&s_bar[b], (done >> 1) & 1u, kWaitPolls)) { bad = true; continue; }
      ++done;
      if (valid) {
#pragma unroll
        for (int m = 0; m < kCompPerBox; ++m)
          if (kCompPerBox * g + m < NQ) {
            if constexpr (TH1)
              component_rhs_xy(P, kCompPerBox * g + m, s_q + b * bfl + m * vol + own, sy, sz, Wxy, Fx, Fy, Fz, dq);
            else
              component_rhs<float, true, TH1>(P, kCompPerBox * g + m, s_q + b * bfl + m * vol + own, 1, sy, sz, th,
                                              Fx, Fy, Fz, dq);
          }
      }
    }
    if (__syncthreads_or(bad)) { bad = true; break; }  // the update runs for every tile of every block, or none
    // ---- k into the buffer the last-but-one group used (every thread has passed the barrier
    //      that issued the last group, so it is free until the next tile's first copy)
    float* const sk = s_q + (done & 1u) * bfl + tid;
    if (valid) {
      const float dt = pr<float>(P).dtau;
#pragma unroll
      for (int n = 0; n < NQ; ++n) sk[n * nthr] = dq[n] * dt;
    }
    // ---- the update (as update_kernel), reading k from shared memory
    const UpdInFused<STAGE> in{uio, L.fstride, L.idx(i + 2, j + 2, k + 2), sk, nthr};
    update_cell<STAGE, LEARNED, false, UpdInFused<STAGE>, true>(P, L, uio, in, i, j, k, tau_out, st, nit,
                                                                  nreg, nfb);
    fence_proxy_async_smem();  // this thread's generic accesses of the buffer before the next copy into it
  }
  if (bad) {  // a copy did not complete in time: let the ones in flight land before the block exits
    for (; done < issued; ++done) mbar_wait(&s_bar[done & 1u], (done >> 1) & 1u, kWaitPolls);
  }
  block_stats(io.status, io.max_speed_bits, io.counters, st | (bad ? ST_TIMEOUT : 0u), amax, nit, nreg, nfb);
}

}  // namespace kt
