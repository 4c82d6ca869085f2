// kt_abi.cu -- host side of libkt: the C ABI declared in include/kt.h.
//
// A context holds one or more events.  Every field array spans all events: component n of
// event e starts at n * gs + base_e (gs = sum of the events' padded sizes), so one persistent
// launch per Runge-Kutta stage can walk a table of (event, tile) work items.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/kt.h"
#include "kt_split.cuh"

using namespace kt;

namespace {

constexpr int KSTAT_WORDS = 12;  // device stats block: status, max speed bits, pad, 3 u64 counters from word 4

struct Shape {
  int x, y, z;
};
// candidate tile shapes of the autotuner (threads per block; x stays 32 so a warp is one x-row)
constexpr Shape kShapes[] = {{32, 4, 2}, {32, 8, 1}, {32, 2, 4}, {32, 1, 8}, {32, 4, 1}, {32, 2, 2}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
// candidates: every shape with a persistent grid (blocks resident at once) and with one block per tile,
// each (mixed precision) as a right-hand-side and an update launch per stage, the update reading
// its inputs directly or staged by TMA, or as one fused launch per stage.  The autotuner times the
// split launches with direct reads (0-11) and, where the context can run them, the fused ones
// (24-35); the TMA-staged update measured slower over a whole step and is selected only by
// kt_set_tuning.
constexpr int kNumBase = 2 * kNumShapes;
constexpr int kNumCandidates = 3 * kNumBase;
constexpr int kFusedFirst = 2 * kNumBase;

struct Ctx {
  kt_options opt;
  Params P;
  int mixed = 0;         // 1: float u, e, p and float stencil
  size_t esz = 8;        // bytes per u/e/p element
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // events
  int nev = 0;
  std::vector<Lattice> lat;
  long long gs = 0;      // component stride of every field array
  size_t max_cells = 0;  // physical cells of the largest event
  std::vector<char> ev_set;
  // device memory
  void* base = nullptr;  // owned allocation (null if caller arena)
  size_t bytes = 0;
  double* q = nullptr;   // 15 components
  double* qs = nullptr;  // 15 components
  float* qf = nullptr;   // mixed mode: FP32 copies of q and qs read by the stencil
  float* qsf = nullptr;
  void* U[3] = {};       // 3 x 4 components
  void* E[2] = {};
  void* Pb[2] = {};
  double* stage = nullptr;  // staging: 18 packed fields of the largest event
  EosSeg<double>* seg_d = nullptr;
  EosSeg<float>* seg_f = nullptr;
  RootSeg* seg_r = nullptr;
  RootSegM* seg_m = nullptr;
  double* d_tau = nullptr;
  unsigned* d_stat = nullptr;
  float* d_mlp = nullptr;
  uint32_t* d_mlp_packed = nullptr;
  Lattice* d_lat = nullptr;
  Tile* d_tiles = nullptr;
  CUtensorMap* d_tmaps = nullptr;  // mixed precision: per event, the 4-d maps of qf (first nev) and qsf
  CUtensorMap* d_umaps = nullptr;  // mixed precision: per event, the kUpdMaps maps of the staged update
  int staged = 0;                  // the update kernels read their inputs staged by TMA
  int fused = 0;                   // one fused launch per stage (right-hand side + update)
  int upd_nbuf = 1;                // staged update: buffers per block (2 on a persistent grid)
  float* reg = nullptr;            // regulation factor of the last step, per cell (diagnostics)
  float* z_net = nullptr;          // learned start: the network's output per cell for the current step
  int grid_mlp = 1;                // blocks of mlp_start_kernel
  int max_tiles = 0;
  // work decomposition
  int shape = 0;
  int ntiles = 0;
  int grid_blocks = 0;    // fused stage kernel (FP64)
  int grid_rhs = 0;       // mixed precision: right-hand-side kernel
  int grid_upd = 0;       // mixed precision: update kernel
  bool tuned = false;
  int cand = 0;
  float tune_ms[kNumCandidates] = {};
  int learned = 0;
  int pi32 = 0;          // KT_STORE_PI_FP32: pi, Pi live in the FP32 array qf (components 4-14)
  int cur = 0, prev = 1, spare = 2;
  double tau = 0.0;
  long long steps = 0;
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};  // 3-step graph per rotation phase
  kt_stats last{};
  char err[512] = {0};
};

int fail(Ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

// NVTX range for the duration of a host call (visible in Nsight timelines; no cost without a tool)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(c, KT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool grids_ok(int nev, const kt_grid* grids) {
  if (nev < 1 || !grids) return false;
  for (int e = 0; e < nev; ++e)
    if (grids[e].nx < 1 || grids[e].ny < 1 || grids[e].neta < 1) return false;
  return true;
}

// padded lattices of all events and the shared component stride
void layout(int nev, const kt_grid* grids, std::vector<Lattice>& lat, long long& gs, size_t& max_cells) {
  lat.resize(nev);
  long long off = 0;
  max_cells = 0;
  for (int e = 0; e < nev; ++e) {
    Lattice& L = lat[e];
    L.nx = grids[e].nx; L.ny = grids[e].ny; L.nz = grids[e].neta;
    L.pitch = (int)align_up((size_t)L.nx + 4, 4);
    L.NY = L.ny + 4;
    L.NZ = L.nz + 4;
    L.plane = (long long)L.pitch * L.NY;
    L.base = off;
    off += (long long)align_up((size_t)(L.plane * L.NZ), 32);
    max_cells = std::max(max_cells, (size_t)L.nx * L.ny * L.nz);
  }
  gs = off;
  for (auto& L : lat) L.fstride = gs;
}

int tiles_for(const std::vector<Lattice>& lat, const Shape& s) {
  long long n = 0;
  for (const auto& L : lat)
    n += (long long)((L.nx + s.x - 1) / s.x) * ((L.ny + s.y - 1) / s.y) * ((L.nz + s.z - 1) / s.z);
  return (int)n;
}

void build_tiles(const std::vector<Lattice>& lat, const Shape& s, std::vector<Tile>& out) {
  out.clear();
  for (int e = 0; e < (int)lat.size(); ++e) {
    const Lattice& L = lat[e];
    // eta fastest: a block of a persistent grid walks a contiguous run of tiles up an eta column
    for (int j = 0; j < L.ny; j += s.y)
      for (int i = 0; i < L.nx; i += s.x)
        for (int k = 0; k < L.nz; k += s.z) out.push_back(Tile{e, i, j, k});
  }
}

size_t state_bytes(const std::vector<Lattice>& lat, long long gs, size_t max_cells, int mixed, int eos_n) {
  const size_t fs = (size_t)gs;
  const size_t es = mixed ? 4 : 8;
  int max_tiles = 0;
  for (const auto& s : kShapes) max_tiles = std::max(max_tiles, tiles_for(lat, s));
  size_t b = 0;
  b += align_up(30 * fs * 8, 256);             // q, qs
  if (mixed) b += align_up(30 * fs * 4, 256);  // FP32 copies of q, qs
  b += align_up(12 * fs * es, 256);            // U[3]
  b += align_up(4 * fs * es, 256);             // E[2], P[2]
  b += align_up(18 * max_cells * 8, 256);      // staging
  b += align_up((size_t)(eos_n > 0 ? eos_n : 1) * sizeof(EosSeg<double>), 256);
  b += align_up((size_t)(eos_n > 0 ? eos_n : 1) * sizeof(EosSeg<float>), 256);
  b += align_up((size_t)(eos_n > 0 ? eos_n : 1) * sizeof(RootSeg), 256);
  b += align_up((size_t)(eos_n > 0 ? eos_n : 1) * sizeof(RootSegM), 256);
  b += 256;                                    // tau
  b += 256;                                    // stats
  b += align_up(KT_MLP_NPARAM * 4, 256);       // MLP weights
  b += align_up(KT_MLP_PACKED_BYTES, 256);     // packed MLP weights
  b += align_up(lat.size() * sizeof(Lattice), 256);
  b += align_up((size_t)max_tiles * sizeof(Tile), 256);
  if (mixed) b += align_up(2 * lat.size() * sizeof(CUtensorMap), 256);
  if (mixed) b += align_up(kUpdMaps * lat.size() * sizeof(CUtensorMap), 256);
  b += align_up(fs * 4, 256);                  // regulation factors
  b += align_up(fs * 4, 256);                  // network outputs (learned start)
  return b;
}

void coef_from(Coef& d, const kt_coef* s) {
  d.kind = s ? s->kind : KT_COEF_CONST;
  d.c0 = s ? s->c0 : 0.0;
  d.c1 = s ? s->c1 : 0.0;
  d.c2 = s ? s->c2 : 1.0;
  d.ln_c0 = (d.c0 > 0.0) ? std::log(d.c0) : -INFINITY;
}

template <typename R>
void fill_pr(PR<R>& o, const Params& P) {
  o.inv_d[0] = (R)(1.0 / P.dx);
  o.inv_d[1] = (R)(1.0 / P.dy);
  o.inv_d[2] = (R)(1.0 / P.deta);
  o.half_inv_d[0] = (R)(0.5 / P.dx);
  o.half_inv_d[1] = (R)(0.5 / P.dy);
  o.half_inv_d[2] = (R)(0.5 / P.deta);
  o.theta = (R)P.theta;
  o.inv_dtau = (R)(1.0 / P.dtau);
  o.dtau = (R)P.dtau;
  o.half_dtau = (R)(0.5 * P.dtau);
  o.rate_max = (R)P.rate_max;
  o.tpp = (R)P.tpp;
  o.rho_max = (R)P.rho_max;
  o.xi0_rho_max = (R)(P.xi0 * P.rho_max);
  o.eos_a = (R)P.eos_a;
  o.eta_c0 = (R)P.eta.c0; o.eta_c1 = (R)P.eta.c1; o.eta_inv_c2 = (R)(1.0 / P.eta.c2); o.eta_ln_c0 = (R)P.eta.ln_c0;
  o.eta_inv_c1 = (R)(1.0 / P.eta.c1);
  o.zeta_c0 = (R)P.zeta.c0; o.zeta_c1 = (R)P.zeta.c1; o.zeta_inv_c2 = (R)(1.0 / P.zeta.c2);
  o.zeta_ln_c0 = (R)P.zeta.ln_c0; o.zeta_inv_c1 = (R)(1.0 / P.zeta.c1);
}

// Per-interval cubic coefficients of the table EOS (see kt_eos in kt.h).
template <typename R>
void build_segments(const kt_eos* eos, std::vector<EosSeg<R>>& out) {
  int n = eos->n;
  out.resize(n);
  for (int i = 0; i + 1 < n; ++i) {
    double e0 = eos->e[i], e1 = eos->e[i + 1];
    double de = e1 - e0;
    double P0 = eos->p[i], P1 = eos->p[i + 1];
    double m0 = eos->cs2[i] * de, m1 = eos->cs2[i + 1] * de;
    double T0 = eos->T[i], T1 = eos->T[i + 1];
    double s0 = eos->cs2[i] * T0 / (e0 + P0) * de, s1 = eos->cs2[i + 1] * T1 / (e1 + P1) * de;
    EosSeg<R> s;
    s.e0 = (R)e0; s.inv_de = (R)(1.0 / de);
    s.P0 = (R)P0; s.mP = (R)m0; s.cP2 = (R)(3.0 * (P1 - P0) - 2.0 * m0 - m1); s.cP3 = (R)(2.0 * (P0 - P1) + m0 + m1);
    s.T0 = (R)T0; s.mT = (R)s0; s.cT2 = (R)(3.0 * (T1 - T0) - 2.0 * s0 - s1); s.cT3 = (R)(2.0 * (T0 - T1) + s0 + s1);
    s.l0 = (R)eos->lndelta[i]; s.dl = (R)(eos->lndelta[i + 1] - eos->lndelta[i]);
    const double c2 = 3.0 * (P1 - P0) - 2.0 * m0 - m1, c3 = 2.0 * (P0 - P1) + m0 + m1;
    s.a1 = (R)(m0 / de); s.a2 = (R)(c2 / (de * de)); s.a3 = (R)(c3 / (de * de * de));
    out[i] = s;
  }
  out[n - 1] = out[n - 2];
  out[n - 1].e0 = (R)eos->e[n - 1];  // sentinel: only its e0 is read by the interval search
}

// The root-find's records (RootSeg) from the FP64 and FP32 segments.
void build_root_segments(const std::vector<EosSeg<double>>& sd, const std::vector<EosSeg<float>>& sf,
                         std::vector<RootSeg>& out) {
  const int n = (int)sd.size();
  out.resize(n);
  for (int i = 0; i < n; ++i) {
    RootSeg r;
    r.e0 = sd[i].e0;
    r.e1 = (i + 2 < n) ? sd[i + 1].e0 : INFINITY;  // the last interval (n - 2) and the sentinel are open
    r.P0 = sd[i].P0;
    r.a1 = sd[i].a1;
    r.a2 = sd[i].a2;
    r.a3 = sd[i].a3;
    const float two = 2.f, three = 3.f;
    r.b1 = sf[i].a1;
    r.b2 = two * sf[i].a2;
    r.b3 = three * sf[i].a3;
    r.unused = 0.f;
    out[i] = r;
  }
}

// The mixed-precision root-find's records: the FP64 ones with a2, a3 rounded to single precision.
void build_mixed_root_segments(const std::vector<RootSeg>& sr, std::vector<RootSegM>& out) {
  out.resize(sr.size());
  for (size_t i = 0; i < sr.size(); ++i) {
    const RootSeg& r = sr[i];
    RootSegM m;
    m.e0 = r.e0;
    m.e1 = r.e1;
    m.P0 = r.P0;
    m.a1 = r.a1;
    m.a2 = (float)r.a2;
    m.a3 = (float)r.a3;
    m.b1 = r.b1;
    m.b2 = r.b2;
    m.b3 = r.b3;
    m.unused0 = m.unused1 = m.unused2 = 0.f;
    out[i] = m;
  }
}

// ------------------------------------------------------------------ small kernels
__device__ __forceinline__ double gnn_at(const Params& P, double tau) { return P.milne ? tau * tau : 1.0; }

// conserved variables from primaries (Eqs. Ttt, Tti) for one event, with its ghost copies
template <typename R>
__global__ void set_state_kernel(const Params P, const Lattice L, const double* __restrict__ in, int has_u, int has_pi,
                                 int has_Pi, int has_up, double tau, double* q, float* qf, R* U, R* Up, R* E, R* Pb,
                                 float* reg, unsigned* status) {
  long long ncp = (long long)L.nx * L.ny * L.nz;
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= ncp) return;
  int i = (int)(o % L.nx), j = (int)((o / L.nx) % L.ny), k = (int)(o / ((long long)L.nx * L.ny));
  const double* pe = in;
  const double* pu = in + ncp;
  const double* ppi = in + 4 * ncp;
  const double* pPi = in + 14 * ncp;
  const double* pup = in + 15 * ncp;
  double e = pe[o];
  double ux = has_u ? pu[o] : 0.0, uy = has_u ? pu[ncp + o] : 0.0, un = has_u ? pu[2 * ncp + o] : 0.0;
  double g = gnn_at(P, tau);
  double ut = sqrt(1.0 + ux * ux + uy * uy + g * un * un);
  double pi[10];
  for (int m = 0; m < 10; ++m) pi[m] = has_pi ? ppi[m * ncp + o] : 0.0;
  double Pi = has_Pi ? pPi[o] : 0.0;
  double P0 = eos_P<double>(P, e);
  double Pt = P0 + Pi;
  double qn[NQ];
  qn[0] = (e + Pt) * ut * ut - Pt + pi[0];
  qn[1] = (e + Pt) * ut * ux + pi[1];
  qn[2] = (e + Pt) * ut * uy + pi[2];
  qn[3] = (e + Pt) * ut * un + pi[3];
  for (int m = 0; m < 10; ++m) qn[4 + m] = pi[m];
  qn[14] = Pi;
  double u4[4] = {ut, ux, uy, un}, up4[4];
  if (has_up) {
    double px = pup[o], py = pup[ncp + o], pn = pup[2 * ncp + o];
    double gp = gnn_at(P, tau - P.dtau);
    up4[0] = sqrt(1.0 + px * px + py * py + gp * pn * pn); up4[1] = px; up4[2] = py; up4[3] = pn;
  } else {
    for (int m = 0; m < 4; ++m) up4[m] = u4[m];
  }
  bool bad = !isfinite(e) || !(e >= 0.0) || !isfinite(ut) || !isfinite(Pi) || !isfinite(up4[0]);
  for (int m = 0; m < 10; ++m) bad |= !isfinite(pi[m]);
  if (bad) atomicOr(status, ST_NONFINITE);
  // the inversion of Eq. (eInferred) needs E = T^{tau tau} - pi^{tau tau} > 0 and M^2 < E^2 with
  // M^i = T^{tau i} - pi^{tau i}, M^2 = M_x^2 + M_y^2 + g_{eta eta} M_eta^2 (Sec. 2.4)
  const double Ei = qn[0] - qn[4], Mx = qn[1] - qn[5], My = qn[2] - qn[6], Mn = qn[3] - qn[7];
  if (!bad && !(Ei > 0.0 && Mx * Mx + My * My + g * Mn * Mn < Ei * Ei)) atomicOr(status, ST_INVERSION);
  const long long fs = L.fstride;
  const int pc[3] = {i + 2, j + 2, k + 2};
  const int nn[3] = {L.nx, L.ny, L.nz};
  reg[L.idx(pc[0], pc[1], pc[2])] = 1.f;  // no regulation recorded yet
  for (int t = -1; t < 12; ++t) {
    int ii = pc[0], jj = pc[1], kk = pc[2];
    if (t >= 0) {
      int ax = t / 4, gi = t % 4, n = nn[ax];
      int gpos = (gi < 2) ? gi : n + gi;
      if (ghost_source(gpos, n, P.periodic) != pc[ax]) continue;
      if (ax == 0) ii = gpos; else if (ax == 1) jj = gpos; else kk = gpos;
    }
    long long c = L.idx(ii, jj, kk);
    for (int n = 0; n < NQ; ++n) q[n * fs + c] = qn[n];
    if (qf)
      for (int n = 0; n < NQ; ++n) qf[n * fs + c] = (float)qn[n];
    for (int m = 0; m < 4; ++m) { U[m * fs + c] = (R)u4[m]; Up[m * fs + c] = (R)up4[m]; }
    E[c] = (R)e;
    Pb[c] = (R)P0;
  }
}

// gather one component of one event (double or float) into a packed physical array
template <typename S>
__global__ void gather_kernel(const Lattice L, const S* __restrict__ f, double* out) {
  long long ncp = (long long)L.nx * L.ny * L.nz;
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= ncp) return;
  int i = (int)(o % L.nx), j = (int)((o / L.nx) % L.ny), k = (int)(o / ((long long)L.nx * L.ny));
  out[o] = (double)f[L.idx(i + 2, j + 2, k + 2)];
}

// scatter one packed physical array into a field (double or float) at every physical cell and
// the ghost copies it owns (checkpoint restore; float fields round to nearest, which is exact
// for values that were float to begin with)
template <typename S>
__global__ void scatter_kernel(const Params P, const Lattice L, const double* __restrict__ in, S* f) {
  long long ncp = (long long)L.nx * L.ny * L.nz;
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= ncp) return;
  int i = (int)(o % L.nx), j = (int)((o / L.nx) % L.ny), k = (int)(o / ((long long)L.nx * L.ny));
  const S v = (S)in[o];
  for_cell_and_ghosts(P, L, i + 2, j + 2, k + 2, [&](long long t) { f[t] = v; });
}

__global__ void advance_tau_kernel(double* tau, double dtau) { tau[0] += dtau; }

// smallest and largest e and smallest regulation factor over one event's physical cells (all
// positive, so their float bit patterns order like the values): out[0] min e, [1] max e, [2] min f
template <typename R>
__global__ void state_extrema_kernel(const Lattice L, const R* __restrict__ e, const float* __restrict__ reg,
                                     unsigned* out) {
  const long long ncp = (long long)L.nx * L.ny * L.nz;
  unsigned lo = 0x7f800000u, hi = 0u, rl = 0x7f800000u;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < ncp; o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % L.nx), j = (int)((o / L.nx) % L.ny), k = (int)(o / ((long long)L.nx * L.ny));
    const long long c = L.idx(i + 2, j + 2, k + 2);
    const unsigned b = __float_as_uint(fmaxf(to_f32(e[c]), 0.f));
    lo = min(lo, b);
    hi = max(hi, b);
    rl = min(rl, __float_as_uint(fmaxf(reg[c], 0.f)));
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  rl = __reduce_min_sync(0xffffffffu, rl);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out, lo);
    atomicMax(out + 1, hi);
    atomicMin(out + 2, rl);
  }
}

// self-test of the integer-pipe double -> float conversions (rounded and truncating)
__global__ void cvt_selftest_kernel(const double* __restrict__ x, float* rn, float* rz, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    rn[i] = d2f_bits(x[i]);
    rz[i] = d2f_trunc(x[i]);
  }
}

// self-test of the FP64 division of the stencil (vdiv) on caller-given operands
__global__ void div_selftest_kernel(const double* __restrict__ a, const double* __restrict__ b, double* q,
                                    long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = vdiv(a[i], b[i]);
}

// Self-test of the bounded waits: every thread waits on an mbarrier that nothing arms, with the
// given poll limit, exactly as the stage kernels wait for their TMA copies; the block records
// ST_TIMEOUT and returns.
__global__ void wait_selftest_kernel(unsigned polls, unsigned* status) {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x == 0) {
    kt::mbar_init(&bar, 1);
    kt::fence_barrier_init();
  }
  __syncthreads();
  const bool ok = kt::mbar_wait(&bar, 0u, polls);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

// validity diagnostics of Sec. 7 at the current state of one event (kt_get_diagnostics): the
// stage-1 right-hand side's kinematics and coefficients, evaluated per physical cell into the
// packed output [7][cells], the last column the recorded regulation factor
template <typename R>
__global__ void diag_kernel(const Params P, const Lattice L, const StageIO<R> io, double tau, const float* reg,
                            double* out) {
  const long long ncp = (long long)L.nx * L.ny * L.nz;
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= ncp) return;
  const int i = (int)(o % L.nx), j = (int)((o / L.nx) % L.ny), k = (int)(o / ((long long)L.nx * L.ny));
  const long long c = L.idx(i + 2, j + 2, k + 2);
  const CellGeom<R> G = cell_geom<R>(P, tau);
  R dq[NQ], du[4][4], dv, dg[6];
  float amax = 0.f;
  Faces<R> Fx, Fy, Fz;
  R uc[4];
  cell_faces<R, false, false>(P, L, io, c, u_global(L, io, c), G, dq, uc, du, dv, amax, Fx, Fy, Fz);
  cell_sources<R, true>(P, L, io, c, G, uc, du, dv, dq, dg);
  for (int m = 0; m < 6; ++m) out[m * ncp + o] = to_f64<R>(dg[m]);
  out[6 * ncp + o] = f2d_bits(reg[c]);
}

// training samples of the learned start: features as the stage kernel forms them, the exact
// FP64 root and the target 10 ln(e / e_conf)
__global__ void mlp_features_kernel(const Params P, const Lattice L, const double* __restrict__ q,
                                    const float* __restrict__ qf, int pi32, double tau, long long n,
                                    const long long* __restrict__ cells, float* X, float* Y, double* Eexact,
                                    unsigned* status) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const long long ncp = (long long)L.nx * L.ny * L.nz;
  const long long o = cells[s];
  if (o < 0 || o >= ncp) {
    atomicOr(status, ST_INVERSION);
    return;
  }
  const int i = (int)(o % L.nx), j = (int)((o / L.nx) % L.ny), k = (int)(o / ((long long)L.nx * L.ny));
  const long long c = L.idx(i + 2, j + 2, k + 2);
  double qn[NQ];
  for (int m = 0; m < NQ; ++m) qn[m] = (pi32 && m >= 4) ? (double)qf[m * L.fstride + c] : q[m * L.fstride + c];
  const float Ef = d2f_bits(qn[0] - qn[4]);
  const double Mx = qn[1] - qn[5], My = qn[2] - qn[6], Mn = qn[3] - qn[7];
  const double g = P.milne ? tau * tau : 1.0;
  const float M2f = d2f_bits(fma(Mx, Mx, fma(My, My, g * Mn * Mn)));
  float x[MLP_IN], ecE;
  mlp_features(fmaxf(Ef, 1e-30f), M2f, d2f_bits(qn[14]), x, ecE);
  double e, P0, uo[4];
  unsigned it = 0;
  const unsigned st = invert_fp64(P, tau, qn, qn[0] - qn[4], e, P0, uo, it);
  if (st) atomicOr(status, st);
  for (int m = 0; m < MLP_IN; ++m) X[s * MLP_IN + m] = x[m];
  Y[s] = (float)(10.0 * log(e / ((double)Ef * (double)ecE)));
  Eexact[s] = e;
}

// ------------------------------------------------------------------ launches
template <typename R>
StageIO<R> make_io(Ctx* c, int stage) {
  StageIO<R> io;
  R* U0 = (R*)c->U[c->cur];
  R* Uprev = (R*)c->U[c->prev];
  R* Usp = (R*)c->U[c->spare];
  if (stage == 1) {
    io.q_in = c->q; io.q_base = nullptr; io.q_out = c->qs;
    io.u_in = U0; io.u_prev = Uprev; io.u_out = Uprev;        // u^* over u^{n-1}
    io.e_in = (R*)c->E[0]; io.p_in = (R*)c->Pb[0];
    io.e_out = (R*)c->E[1]; io.p_out = (R*)c->Pb[1];
  } else {
    io.q_in = c->qs; io.q_base = c->q; io.q_out = c->q;       // q^{n+1} over q^n
    io.u_in = Uprev; io.u_prev = U0; io.u_out = Usp;          // u^{n+1} into the spare buffer
    io.e_in = (R*)c->E[1]; io.p_in = (R*)c->Pb[1];
    io.e_out = (R*)c->E[0]; io.p_out = (R*)c->Pb[0];
  }
  if constexpr (sizeof(R) == 4) {
    io.qr_in = (stage == 1) ? c->qf : c->qsf;
    io.qr_out = (stage == 1) ? c->qsf : c->qf;
  } else {
    io.qr_in = (const R*)io.q_in;
    io.qr_out = nullptr;
  }
  io.d_tau = c->d_tau;
  io.status = c->d_stat;
  io.max_speed_bits = c->d_stat + 1;
  io.counters = (unsigned long long*)(c->d_stat + 4);
  io.mlp_packed = c->learned ? c->d_mlp_packed : nullptr;
  io.reg_out = (stage == 2) ? c->reg : nullptr;
  return io;
}

// Mixed precision: the Runge-Kutta increments k_1, k_2 (FP32, 15 components each) live in the
// memory of the FP64 q* array, which that path never stores.
float* k_buf(Ctx* c, int stage) { return (float*)c->qs + (stage == 1 ? 0 : 15 * c->gs); }

UpdIO make_uio(Ctx* c, int stage) {
  UpdIO u;
  StageIO<float> io = make_io<float>(c, stage);
  u.q = c->q;
  u.qf_n = c->qf;
  u.qsf = c->qsf;
  u.k1 = k_buf(c, 1);
  u.k2 = k_buf(c, 2);
  u.qr_out = io.qr_out;
  u.u_out = io.u_out;
  u.e_out = io.e_out;
  u.p_out = io.p_out;
  u.e_guess = io.e_in;
  u.d_tau = c->d_tau;
  u.status = c->d_stat;
  u.counters = (unsigned long long*)(c->d_stat + 4);
  u.reg_out = io.reg_out;
  u.z_net = c->z_net;
  return u;
}

template <int STAGE>
void launch_stage(Ctx* c, const StageIO<double>& io) {
  const Shape& s = kShapes[c->shape];
  const dim3 blk(s.x, s.y, s.z);
  const bool t1 = (c->P.theta == 1.0), inv = c->P.iface_invert;
  if (t1 && !inv)
    stage_kernel<double, STAGE, true, false><<<c->grid_blocks, blk, 0, c->stream>>>(c->P, io, c->d_lat, c->d_tiles, c->ntiles);
  else if (!inv)
    stage_kernel<double, STAGE, false, false><<<c->grid_blocks, blk, 0, c->stream>>>(c->P, io, c->d_lat, c->d_tiles, c->ntiles);
  else if (t1)
    stage_kernel<double, STAGE, true, true><<<c->grid_blocks, blk, 0, c->stream>>>(c->P, io, c->d_lat, c->d_tiles, c->ntiles);
  else
    stage_kernel<double, STAGE, false, true><<<c->grid_blocks, blk, 0, c->stream>>>(c->P, io, c->d_lat, c->d_tiles, c->ntiles);
}

// the right-hand-side kernel of a stage, with the minmod specialised when theta = 1
template <int STAGE>
void launch_rhs(Ctx* c, const StageIO<float>& io) {
  const Shape& s = kShapes[c->shape];
  const dim3 blk(s.x, s.y, s.z);
  const CUtensorMap* maps = c->d_tmaps + (STAGE == 1 ? 0 : c->nev);
  const size_t sm = rhs_smem_bytes(s.x, s.y, s.z);
  float* k = k_buf(c, STAGE);
  const bool t1 = (c->P.theta == 1.0), inv = c->P.iface_invert;
  if (t1 && !inv)
    rhs_kernel<STAGE, true, false><<<c->grid_rhs, blk, sm, c->stream>>>(c->P, io, k, c->d_lat, c->d_tiles, c->ntiles, maps);
  else if (!inv)
    rhs_kernel<STAGE, false, false><<<c->grid_rhs, blk, sm, c->stream>>>(c->P, io, k, c->d_lat, c->d_tiles, c->ntiles, maps);
  else if (t1)
    rhs_kernel<STAGE, true, true><<<c->grid_rhs, blk, sm, c->stream>>>(c->P, io, k, c->d_lat, c->d_tiles, c->ntiles, maps);
  else
    rhs_kernel<STAGE, false, true><<<c->grid_rhs, blk, sm, c->stream>>>(c->P, io, k, c->d_lat, c->d_tiles, c->ntiles, maps);
}

// every rhs kernel may take the dynamic shared memory of the largest tile shape
int allow_rhs_smem(Ctx* c) {
  int bytes = 0;
  for (const auto& sh : kShapes) bytes = std::max(bytes, rhs_smem_bytes(sh.x, sh.y, sh.z));
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)rhs_kernel<1, true, false>);
  set((const void*)rhs_kernel<1, false, false>);
  set((const void*)rhs_kernel<1, true, true>);
  set((const void*)rhs_kernel<1, false, true>);
  set((const void*)rhs_kernel<2, true, false>);
  set((const void*)rhs_kernel<2, false, false>);
  set((const void*)rhs_kernel<2, true, true>);
  set((const void*)rhs_kernel<2, false, true>);
  set((const void*)fused_kernel<1, true, false, true>);
  set((const void*)fused_kernel<1, true, false, false>);
  set((const void*)fused_kernel<1, false, false, true>);
  set((const void*)fused_kernel<1, false, false, false>);
  set((const void*)fused_kernel<2, true, false, true>);
  set((const void*)fused_kernel<2, true, false, false>);
  set((const void*)fused_kernel<2, false, false, true>);
  set((const void*)fused_kernel<2, false, false, false>);
  if (e != cudaSuccess) return fail(c, KT_ERR_CUDA, "rhs shared memory: %s", cudaGetErrorString(e));
  bytes = 0;
  for (const auto& sh : kShapes) bytes = std::max(bytes, upd_smem_bytes(sh.x, sh.y, sh.z, 2));
  set((const void*)update_staged_kernel<1, true>);
  set((const void*)update_staged_kernel<1, false>);
  set((const void*)update_staged_kernel<2, true>);
  set((const void*)update_staged_kernel<2, false>);
  if (e != cudaSuccess) return fail(c, KT_ERR_CUDA, "update shared memory: %s", cudaGetErrorString(e));
  return KT_OK;
}

// the update kernel of a stage for the context's root-find start and pi storage
template <int STAGE>
void launch_update(Ctx* c, const UpdIO& uio) {
  const Shape& s = kShapes[c->shape];
  const dim3 blk(s.x, s.y, s.z);
  if (c->staged && !c->pi32) {
    const size_t sm = upd_smem_bytes(s.x, s.y, s.z, c->upd_nbuf);
    if (c->learned)
      update_staged_kernel<STAGE, true><<<c->grid_upd, blk, sm, c->stream>>>(c->P, uio, c->d_lat, c->d_tiles,
                                                                             c->ntiles, c->d_umaps, c->upd_nbuf);
    else
      update_staged_kernel<STAGE, false><<<c->grid_upd, blk, sm, c->stream>>>(c->P, uio, c->d_lat, c->d_tiles,
                                                                              c->ntiles, c->d_umaps, c->upd_nbuf);
    return;
  }
  if (c->learned && c->pi32)
    update_kernel<STAGE, true, true><<<c->grid_upd, blk, 0, c->stream>>>(c->P, uio, c->d_lat, c->d_tiles, c->ntiles);
  else if (c->learned)
    update_kernel<STAGE, true, false><<<c->grid_upd, blk, 0, c->stream>>>(c->P, uio, c->d_lat, c->d_tiles, c->ntiles);
  else if (c->pi32)
    update_kernel<STAGE, false, true><<<c->grid_upd, blk, 0, c->stream>>>(c->P, uio, c->d_lat, c->d_tiles, c->ntiles);
  else
    update_kernel<STAGE, false, false><<<c->grid_upd, blk, 0, c->stream>>>(c->P, uio, c->d_lat, c->d_tiles, c->ntiles);
}

// the fused stage kernel (right-hand side and update in one launch)
template <int STAGE>
void launch_fused(Ctx* c, const StageIO<float>& io, const UpdIO& uio) {
  const Shape& s = kShapes[c->shape];
  const dim3 blk(s.x, s.y, s.z);
  const CUtensorMap* maps = c->d_tmaps + (STAGE == 1 ? 0 : c->nev);
  const size_t sm = rhs_smem_bytes(s.x, s.y, s.z);
  const bool t1 = (c->P.theta == 1.0);
  if (t1 && c->learned)
    fused_kernel<STAGE, true, false, true><<<c->grid_rhs, blk, sm, c->stream>>>(c->P, io, uio, c->d_lat, c->d_tiles,
                                                                               c->ntiles, maps);
  else if (t1)
    fused_kernel<STAGE, true, false, false><<<c->grid_rhs, blk, sm, c->stream>>>(c->P, io, uio, c->d_lat, c->d_tiles,
                                                                                c->ntiles, maps);
  else if (c->learned)
    fused_kernel<STAGE, false, false, true><<<c->grid_rhs, blk, sm, c->stream>>>(c->P, io, uio, c->d_lat, c->d_tiles,
                                                                                c->ntiles, maps);
  else
    fused_kernel<STAGE, false, false, false><<<c->grid_rhs, blk, sm, c->stream>>>(c->P, io, uio, c->d_lat, c->d_tiles,
                                                                                 c->ntiles, maps);
}

template <int STAGE>
void launch_split_stage(Ctx* c, const StageIO<float>& io, const UpdIO& uio) {
  if (c->fused) {
    launch_fused<STAGE>(c, io, uio);
    return;
  }
  launch_rhs<STAGE>(c, io);
  launch_update<STAGE>(c, uio);
}

// ev (optional, kNumTimed + 1 events): recorded between the launches of one step, in the order
// learned start (the network's inference), stage-1 rhs (or fused stage 1), stage-1 update,
// stage-2 rhs (or fused stage 2), stage-2 update, tau advance; intervals of launches a context
// does not make (the network without the learned start, the update launches of the FP64 path and
// of the fused layout) are empty.
constexpr int kNumTimed = 6;
void mark(Ctx* c, cudaEvent_t* ev, int i) {
  if (ev) cudaEventRecord(ev[i], c->stream);
}

// the learned start's network on the state at the start of the step (its FP32 copy)
void launch_mlp_start(Ctx* c) {
  kt::mlp_start_kernel<<<c->grid_mlp, 256, 0, c->stream>>>(c->qf, c->gs, c->d_tau, c->P.milne,
                                                           c->d_mlp_packed, c->z_net);
}

template <typename R>
void launch_step_stages(Ctx* c, cudaEvent_t* ev) {
  mark(c, ev, 0);
  if constexpr (sizeof(R) == 4) {
    if (c->learned && c->P.mlp_infer) launch_mlp_start(c);
    mark(c, ev, 1);
    if (c->fused) {  // the fused launches take the right-hand-side slots; the update slots stay empty
      launch_fused<1>(c, make_io<float>(c, 1), make_uio(c, 1));
      mark(c, ev, 2);
      mark(c, ev, 3);
      launch_fused<2>(c, make_io<float>(c, 2), make_uio(c, 2));
      mark(c, ev, 4);
      mark(c, ev, 5);
      return;
    }
    launch_rhs<1>(c, make_io<float>(c, 1));
    mark(c, ev, 2);
    launch_update<1>(c, make_uio(c, 1));
    mark(c, ev, 3);
    launch_rhs<2>(c, make_io<float>(c, 2));
    mark(c, ev, 4);
    launch_update<2>(c, make_uio(c, 2));
    mark(c, ev, 5);
  } else {
    mark(c, ev, 1);
    launch_stage<1>(c, make_io<double>(c, 1));
    mark(c, ev, 2);
    mark(c, ev, 3);
    launch_stage<2>(c, make_io<double>(c, 2));
    mark(c, ev, 4);
    mark(c, ev, 5);
  }
}

// enqueue one full step (two stages + tau advance) for the current rotation phase, then rotate
int enqueue_step(Ctx* c, cudaEvent_t* ev = nullptr) {
  if (c->mixed) launch_step_stages<float>(c, ev);
  else launch_step_stages<double>(c, ev);
  advance_tau_kernel<<<1, 1, 0, c->stream>>>(c->d_tau, c->P.dtau);
  mark(c, ev, 6);
  // u^{n-1} <- u^n, u^n <- u^{n+1}; the old u^{n-1} buffer (holding u^*) becomes the spare
  int ncur = c->spare, nprev = c->cur, nspare = c->prev;
  c->cur = ncur; c->prev = nprev; c->spare = nspare;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, KT_ERR_CUDA, "stage launch: %s", cudaGetErrorString(e));
  return KT_OK;
}

// persistent grid: as many blocks of kernel K as fit on the device at once
template <typename K>
int occupancy_blocks(K kernel, const Shape& s, size_t dyn_smem = 0) {
  int nb = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, s.x * s.y * s.z, dyn_smem);
  return std::max(1, nb) * std::max(1, sms);
}

// The TMA descriptors of the FP32 copies of q read by the mixed-precision stencil: per event a
// 4-d map (x: pitch, y: ny + 4, eta: neta + 4, component: 15) with the strides of the padded
// lattice, and a box of the tile plus its two-cell halo for kCompPerBox components,
// (bx + 4) x (by + 4) x (bz + 4) x kCompPerBox.
int encode_tensor_maps(Ctx* c) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(c, KT_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const Shape& s = kShapes[c->shape];
  if ((s.x + 4) * (s.y + 4) * (s.z + 4) > kBoxMax) return fail(c, KT_ERR_ARG, "tile box exceeds the staging buffer");
  std::vector<CUtensorMap> maps(2 * c->nev);
  for (int w = 0; w < 2; ++w)
    for (int e = 0; e < c->nev; ++e) {
      const Lattice& L = c->lat[e];
      float* base = (w == 0 ? c->qf : c->qsf) + L.base;
      cuuint64_t dims[4] = {(cuuint64_t)L.pitch, (cuuint64_t)L.NY, (cuuint64_t)L.NZ, (cuuint64_t)NQ};
      cuuint64_t strides[3] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4, (cuuint64_t)c->gs * 4};
      cuuint32_t box[4] = {(cuuint32_t)(s.x + 4), (cuuint32_t)(s.y + 4), (cuuint32_t)(s.z + 4), kCompPerBox};
      cuuint32_t estr[4] = {1, 1, 1, 1};
      CUresult r = encode(&maps[w * c->nev + e], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(c, KT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for event %d", (int)r, e);
    }
  CK(cudaMemcpyAsync(c->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, c->stream));
  // the staged update's boxes: the tile's cells in y and eta, bx + 4 cells in x from the tile's
  // padded x, for q (FP64: 8 components, and 1), k_1, k_2 and the FP32 copy of q (15 components)
  std::vector<CUtensorMap> um(kUpdMaps * c->nev);
  for (int e = 0; e < c->nev; ++e) {
    const Lattice& L = c->lat[e];
    struct Src { void* base; CUtensorMapDataType t; int esz; cuuint32_t depth; };
    const Src src[kUpdMaps] = {{c->q + L.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, 8},
                               {c->q + L.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, 1},
                               {k_buf(c, 1) + L.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, NQ},
                               {k_buf(c, 2) + L.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, NQ},
                               {c->qf + L.base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, NQ}};
    for (int w = 0; w < kUpdMaps; ++w) {
      const cuuint64_t es = (cuuint64_t)src[w].esz;
      cuuint64_t dims[4] = {(cuuint64_t)L.pitch, (cuuint64_t)L.NY, (cuuint64_t)L.NZ, (cuuint64_t)NQ};
      cuuint64_t strides[3] = {(cuuint64_t)L.pitch * es, (cuuint64_t)L.plane * es, (cuuint64_t)c->gs * es};
      cuuint32_t box[4] = {(cuuint32_t)(s.x + 4), (cuuint32_t)s.y, (cuuint32_t)s.z, src[w].depth};
      cuuint32_t estr[4] = {1, 1, 1, 1};
      CUresult r = encode(&um[kUpdMaps * e + w], src[w].t, 4, src[w].base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return fail(c, KT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d), update map %d", (int)r, w);
    }
  }
  CK(cudaMemcpyAsync(c->d_umaps, um.data(), um.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return KT_OK;
}

int select_shape(Ctx* c, int cand) {
  const int base = cand % kNumBase, shape = base / 2, one_per_tile = base % 2, variant = cand / kNumBase;
  const bool fusable = c->mixed && !c->pi32 && !c->P.iface_invert;
  c->staged = (variant == 1) && c->mixed && !c->pi32;
  c->fused = (variant == 2) && fusable;
  c->upd_nbuf = one_per_tile ? 1 : 2;
  std::vector<Tile> tiles;
  build_tiles(c->lat, kShapes[shape], tiles);
  if ((int)tiles.size() > c->max_tiles) return fail(c, KT_ERR_OOM, "tile table overflow");
  CK(cudaMemcpyAsync(c->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->shape = shape;
  c->ntiles = (int)tiles.size();
  if (c->mixed) {
    int rc = encode_tensor_maps(c);
    if (rc != KT_OK) return rc;
  }
  const Shape& sh = kShapes[shape];
  auto grid = [&](int cap) { return one_per_tile ? c->ntiles : std::max(1, std::min(cap, c->ntiles)); };
  if (c->mixed) {
    const size_t rsm = rhs_smem_bytes(sh.x, sh.y, sh.z);
    c->grid_rhs = grid(c->fused ? occupancy_blocks(fused_kernel<1, true, false, true>, sh, rsm)
                                : occupancy_blocks(rhs_kernel<1, true, false>, sh, rsm));
    if (c->staged) {
      const size_t usm = upd_smem_bytes(sh.x, sh.y, sh.z, c->upd_nbuf);
      c->grid_upd = grid(c->learned ? occupancy_blocks(update_staged_kernel<2, true>, sh, usm)
                                    : occupancy_blocks(update_staged_kernel<2, false>, sh, usm));
    } else {
      c->grid_upd = grid(c->learned ? occupancy_blocks(update_kernel<1, true, false>, sh)
                                    : occupancy_blocks(update_kernel<1, false, false>, sh));
    }
    c->grid_blocks = c->grid_rhs;
  } else {
    c->grid_blocks = grid(occupancy_blocks(stage_kernel<double, 1, true, false>, sh));  // same launch bounds
  }
  c->cand = cand;
  for (int p = 0; p < 3; ++p)
    if (c->graph[p]) { cudaGraphExecDestroy(c->graph[p]); c->graph[p] = nullptr; }
  return KT_OK;
}

// Autotuner: time first-stage launches for every candidate (tile shape, grid size, layout).  The
// launches write only scratch buffers (q*, its FP32 copy, e*, p*, and u* redirected to the spare
// buffer), so the state is untouched; the fastest candidate is kept.
template <typename R>
int time_first_stage(Ctx* c, float* ms) {
  StageIO<R> io = make_io<R>(c, 1);
  io.u_out = (R*)c->U[c->spare];
  auto launch = [&]() {
    if constexpr (sizeof(R) == 4) {  // writes k_1, q*'s FP32 copy, e*, P*, u* (spare buffer)
      UpdIO u = make_uio(c, 1);
      u.u_out = (float*)c->U[c->spare];
      launch_split_stage<1>(c, io, u);
    } else {
      launch_stage<1>(c, io);
    }
  };
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  launch();  // warm-up
  for (int r = 0; r < 3; ++r) {  // the fastest of three timed launches (candidates differ by ~1%)
    CK(cudaEventRecord(a, c->stream));
    launch();
    CK(cudaEventRecord(b, c->stream));
    CK(cudaEventSynchronize(b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, a, b));
    if (r == 0 || t < *ms) *ms = t;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return KT_OK;
}

int autotune(Ctx* c) {
  Range range_("kt autotune");
  int best = 0;
  for (int s = 0; s < kNumCandidates; ++s) c->tune_ms[s] = 0.f;
  const bool fusable = c->mixed && !c->pi32 && !c->P.iface_invert;
  for (int s = 0; s < kNumCandidates; ++s) {
    if (!(s < kNumBase || (fusable && s >= kFusedFirst))) continue;
    int rc = select_shape(c, s);
    if (rc != KT_OK) return rc;
    float ms = 0.f;
    if (c->mixed) rc = time_first_stage<float>(c, &ms);
    else rc = time_first_stage<double>(c, &ms);
    if (rc != KT_OK) return rc;
    c->tune_ms[s] = ms;
    if (ms < c->tune_ms[best]) best = s;
  }
  int rc = select_shape(c, best);
  if (rc != KT_OK) return rc;
  CK(cudaMemsetAsync(c->d_stat, 0, 256, c->stream));
  c->tuned = true;
  return KT_OK;
}

int build_graph(Ctx* c, int phase) {
  Range range_("kt capture step graph");
  int save[3] = {c->cur, c->prev, c->spare};
  cudaGraph_t gr;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int rc = KT_OK;
  for (int s = 0; s < 3 && rc == KT_OK; ++s) rc = enqueue_step(c);
  cudaError_t e = cudaStreamEndCapture(c->stream, &gr);
  c->cur = save[0]; c->prev = save[1]; c->spare = save[2];
  if (rc != KT_OK) return rc;
  if (e != cudaSuccess) return fail(c, KT_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->graph[phase], gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(c, KT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return KT_OK;
}

}  // namespace

struct kt_ctx : Ctx {};

// ==================================================================== C ABI
extern "C" {

int kt_options_default(kt_options* o) {
  if (!o) return KT_ERR_ARG;
  memset(o, 0, sizeof(*o));
  o->theta_limiter = 1.0;
  o->coords = KT_MILNE;
  o->bc = KT_BC_COPY;
  o->precision = KT_FP64;
  o->inversion = KT_INV_PLAIN;
  o->tau_pipi_on = 1;
  o->regulate = 1;
  o->rho_max = 1.0;
  o->xi0 = 0.1;
  o->e_min = 0.0;
  o->tau_relax_min = 0.0;
  o->use_graph = 1;
  o->autotune = 1;
  o->iface = KT_IFACE_RECON;
  return KT_OK;
}

int kt_state_bytes_batch(int n_events, const kt_grid* grids, const kt_eos* eos, const kt_options* opt,
                         size_t* bytes) {
  if (!bytes || !grids_ok(n_events, grids)) return KT_ERR_ARG;
  if (eos && eos->kind == KT_EOS_TABLE && eos->n < 4) return KT_ERR_EOS;
  kt_options d;
  kt_options_default(&d);
  const kt_options* o = opt ? opt : &d;
  std::vector<Lattice> lat;
  long long gs;
  size_t mc;
  layout(n_events, grids, lat, gs, mc);
  *bytes = state_bytes(lat, gs, mc, o->precision == KT_MIXED, (eos && eos->kind == KT_EOS_TABLE) ? eos->n : 0);
  return KT_OK;
}

int kt_state_bytes(const kt_grid* grid, const kt_eos* eos, const kt_options* opt, size_t* bytes) {
  return kt_state_bytes_batch(1, grid, eos, opt, bytes);
}

int kt_init_batch(kt_ctx** out, int n_events, const kt_grid* grids, double dx, double deta, double dtau,
                  const kt_eos* eos, const kt_coef* eta_over_s, const kt_coef* zeta_over_s, const kt_options* opt) {
  if (!out) return KT_ERR_ARG;
  *out = nullptr;
  kt_ctx* c = new (std::nothrow) kt_ctx();
  if (!c) return KT_ERR_OOM;
  auto bail = [&](int code) { kt_free(c); return code; };
  if (!grids_ok(n_events, grids) || !(dx > 0) || !(deta > 0) || !(dtau > 0) || !eos) {
    fprintf(stderr, "kt_init: invalid grid, spacing or eos\n");
    return bail(KT_ERR_ARG);
  }
  if (opt) c->opt = *opt; else kt_options_default(&c->opt);
  const kt_options& o = c->opt;
  if (o.precision != KT_FP64 && o.precision != KT_MIXED) return bail(KT_ERR_ARG);
  if (!(o.theta_limiter >= 1.0 && o.theta_limiter <= 2.0)) return bail(KT_ERR_ARG);
  if (o.coords != KT_MILNE && o.coords != KT_CARTESIAN) return bail(KT_ERR_ARG);
  if (o.bc != KT_BC_COPY && o.bc != KT_BC_PERIODIC) return bail(KT_ERR_ARG);
  if (o.inversion != KT_INV_PLAIN && o.inversion != KT_INV_LEARNED && o.inversion != KT_INV_CONFORMAL)
    return bail(KT_ERR_ARG);
  // the learned (and the conformal) start serves the mixed-precision path
  if (o.inversion == KT_INV_LEARNED && (!o.mlp_weights || o.precision != KT_MIXED)) return bail(KT_ERR_ARG);
  if (o.inversion == KT_INV_CONFORMAL && o.precision != KT_MIXED) return bail(KT_ERR_ARG);
  c->mixed = (o.precision == KT_MIXED);
  c->esz = c->mixed ? 4 : 8;
  c->learned = (o.inversion == KT_INV_LEARNED || o.inversion == KT_INV_CONFORMAL);
  if (o.pi_storage != KT_STORE_FP64 && o.pi_storage != KT_STORE_PI_FP32) return bail(KT_ERR_ARG);
  if (o.pi_storage == KT_STORE_PI_FP32 && o.precision != KT_MIXED) return bail(KT_ERR_ARG);
  c->pi32 = (o.pi_storage == KT_STORE_PI_FP32);
  c->nev = n_events;
  layout(n_events, grids, c->lat, c->gs, c->max_cells);
  c->ev_set.assign(n_events, 0);

  Params& P = c->P;
  memset(&P, 0, sizeof(P));
  P.dx = dx; P.dy = dx; P.deta = deta; P.dtau = dtau;
  P.theta = o.theta_limiter;
  P.milne = (o.coords == KT_MILNE);
  P.periodic = (o.bc == KT_BC_PERIODIC);
  coef_from(P.eta, eta_over_s);
  coef_from(P.zeta, zeta_over_s);
  for (const Coef* k : {&P.eta, &P.zeta}) {
    const bool ok = (k->kind == KT_COEF_CONST && k->c0 >= 0.0) ||
                    (k->kind == KT_COEF_GAUSS && k->c0 >= 0.0 && k->c2 > 0.0) ||
                    (k->kind == KT_COEF_PAPER_ZETA && k->c0 >= 0.0 && k->c1 > 0.0);
    if (!ok) return bail(KT_ERR_ARG);
  }
  P.eos_table = (eos->kind == KT_EOS_TABLE);
  P.eos_a = eos->a;
  if (eos->kind == KT_EOS_TABLE) {
    if (eos->n < 4 || !eos->e || !eos->p || !eos->cs2 || !eos->T || !eos->lndelta) return bail(KT_ERR_EOS);
    for (int i = 0; i + 1 < eos->n; ++i)
      if (!(eos->e[i + 1] > eos->e[i]) || !(eos->e[i] > 0)) return bail(KT_ERR_EOS);
    P.eos_n = eos->n;
    P.lne0 = (float)std::log(eos->e[0]);
    P.inv_h = (float)((eos->n - 1) / (std::log(eos->e[eos->n - 1]) - std::log(eos->e[0])));
  } else if (eos->kind == KT_EOS_CONFORMAL) {
    if (!(eos->a > 0)) return bail(KT_ERR_EOS);
    P.eos_n = 0;
  } else {
    return bail(KT_ERR_EOS);
  }
  P.shear_on = !(P.eta.kind == KT_COEF_CONST && P.eta.c0 == 0.0);
  P.bulk_on = !(P.zeta.kind == KT_COEF_CONST && P.zeta.c0 == 0.0) && P.eos_table;
  P.tpp = o.tau_pipi_on ? 10.0 / 7.0 : 0.0;
  P.regulate = o.regulate;
  if (o.iface != KT_IFACE_RECON && o.iface != KT_IFACE_INVERT) return bail(KT_ERR_ARG);
  P.iface_invert = (o.iface == KT_IFACE_INVERT);
  P.mlp_infer = (o.inversion == KT_INV_LEARNED);
  P.rho_max = o.rho_max;
  P.xi0 = o.xi0;
  P.e_min = o.e_min;
  P.rate_max = (o.tau_relax_min > 0) ? 1.0 / o.tau_relax_min : INFINITY;
  P.ln_rate_max = std::log(P.rate_max);
  fill_pr<double>(P.pd, P);
  fill_pr<float>(P.pf, P);

  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
    fail(c, KT_ERR_CUDA, "no CUDA device");
    fprintf(stderr, "kt_init: no CUDA device (libkt has no CPU fallback)\n");
    return bail(KT_ERR_CUDA);
  }
  // every call synchronises its stream before returning, so a context-owned stream is safe when
  // the caller passes none (the legacy default stream cannot be captured into a graph)
  c->stream = (cudaStream_t)o.stream;
  if (!c->stream) {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      fail(c, KT_ERR_CUDA, "stream creation failed");
      return bail(KT_ERR_CUDA);
    }
    c->own_stream = true;
  }

  // ---- device memory, carved from one block
  size_t need = state_bytes(c->lat, c->gs, c->max_cells, c->mixed, P.eos_n);
  char* base;
  if (o.arena) {
    if (o.arena_bytes < need) return bail(KT_ERR_OOM);
    base = (char*)o.arena;
  } else {
    if (cudaMalloc(&c->base, need) != cudaSuccess) { cudaGetLastError(); return bail(KT_ERR_OOM); }
    base = (char*)c->base;
  }
  c->bytes = need;
  size_t off = 0;
  auto carve = [&](size_t b) { void* p = base + off; off += align_up(b, 256); return p; };
  const size_t fs = (size_t)c->gs;
  char* qq = (char*)carve(30 * fs * 8);
  c->q = (double*)qq;
  c->qs = (double*)(qq + 15 * fs * 8);
  if (c->mixed) {
    char* qqf = (char*)carve(30 * fs * 4);
    c->qf = (float*)qqf;
    c->qsf = (float*)(qqf + 15 * fs * 4);
    CK(cudaMemsetAsync(qqf, 0, 30 * fs * 4, c->stream));
  }
  char* uu = (char*)carve(12 * fs * c->esz);
  for (int b = 0; b < 3; ++b) c->U[b] = uu + (size_t)b * 4 * fs * c->esz;
  char* ep = (char*)carve(4 * fs * c->esz);
  c->E[0] = ep; c->E[1] = ep + fs * c->esz; c->Pb[0] = ep + 2 * fs * c->esz; c->Pb[1] = ep + 3 * fs * c->esz;
  c->stage = (double*)carve(18 * c->max_cells * 8);
  int nseg = P.eos_n > 0 ? P.eos_n : 1;
  c->seg_d = (EosSeg<double>*)carve(nseg * sizeof(EosSeg<double>));
  c->seg_f = (EosSeg<float>*)carve(nseg * sizeof(EosSeg<float>));
  c->seg_r = (RootSeg*)carve(nseg * sizeof(RootSeg));
  c->seg_m = (RootSegM*)carve(nseg * sizeof(RootSegM));
  c->d_tau = (double*)carve(256);
  c->d_stat = (unsigned*)carve(256);
  c->d_mlp = (float*)carve(KT_MLP_NPARAM * 4);
  c->d_mlp_packed = (uint32_t*)carve(KT_MLP_PACKED_BYTES);
  c->d_lat = (Lattice*)carve(c->lat.size() * sizeof(Lattice));
  for (const auto& s : kShapes) c->max_tiles = std::max(c->max_tiles, tiles_for(c->lat, s));
  c->d_tiles = (Tile*)carve((size_t)c->max_tiles * sizeof(Tile));
  if (c->mixed) c->d_tmaps = (CUtensorMap*)carve(2 * c->lat.size() * sizeof(CUtensorMap));
  if (c->mixed) c->d_umaps = (CUtensorMap*)carve(kUpdMaps * c->lat.size() * sizeof(CUtensorMap));
  c->reg = (float*)carve(fs * 4);
  c->z_net = (float*)carve(fs * 4);
  CK(cudaMemsetAsync(c->z_net, 0, fs * 4, c->stream));  // z = 0: the conformal start (no network)
  {
    int nb = 0, dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kt::mlp_start_kernel, 256, 0));
    c->grid_mlp = (int)std::max(1LL, std::min((long long)std::max(1, nb) * sms, (long long)((fs + 255) / 256)));
  }
  P.seg_d = c->seg_d;
  P.seg_f = c->seg_f;
  P.seg_r = c->seg_r;
  P.seg_m = c->seg_m;

  CK(cudaMemsetAsync(qq, 0, 30 * fs * 8, c->stream));
  CK(cudaMemsetAsync(ep, 0, 4 * fs * c->esz, c->stream));
  {  // unused corner ghosts hold a fluid at rest (u^tau = 1); they are never read
    std::vector<unsigned char> one(fs * c->esz, 0);
    for (size_t i = 0; i < fs; ++i) {
      if (c->mixed) { float v = 1.f; memcpy(&one[i * 4], &v, 4); }
      else { double v = 1.0; memcpy(&one[i * 8], &v, 8); }
    }
    for (int b = 0; b < 3; ++b) {
      CK(cudaMemcpyAsync(c->U[b], one.data(), one.size(), cudaMemcpyHostToDevice, c->stream));
      CK(cudaMemsetAsync((char*)c->U[b] + fs * c->esz, 0, 3 * fs * c->esz, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
  }
  if (P.eos_table) {
    std::vector<EosSeg<double>> sd;
    std::vector<EosSeg<float>> sf;
    build_segments<double>(eos, sd);
    build_segments<float>(eos, sf);
    std::vector<RootSeg> sr;
    build_root_segments(sd, sf, sr);
    std::vector<RootSegM> sm;
    build_mixed_root_segments(sr, sm);
    CK(cudaMemcpyAsync(c->seg_d, sd.data(), sd.size() * sizeof(sd[0]), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->seg_f, sf.data(), sf.size() * sizeof(sf[0]), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->seg_r, sr.data(), sr.size() * sizeof(sr[0]), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->seg_m, sm.data(), sm.size() * sizeof(sm[0]), cudaMemcpyHostToDevice, c->stream));
  }
  if (o.mlp_weights) {
    CK(cudaMemcpyAsync(c->d_mlp, o.mlp_weights, KT_MLP_NPARAM * 4, cudaMemcpyHostToDevice, c->stream));
    kt::mlp_pack_kernel<<<1, 256, 0, c->stream>>>(c->d_mlp, c->d_mlp_packed);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(c->d_lat, c->lat.data(), c->lat.size() * sizeof(Lattice), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->d_stat, 0, 256, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int rc = c->mixed ? allow_rhs_smem(c) : KT_OK;
  if (rc == KT_OK) rc = select_shape(c, 0);
  if (rc != KT_OK) return bail(rc);
  *out = c;
  return KT_OK;
}

int kt_init(kt_ctx** out, const kt_grid* grid, double dx, double deta, double dtau, const kt_eos* eos,
            const kt_coef* eta_over_s, const kt_coef* zeta_over_s, const kt_options* opt) {
  return kt_init_batch(out, 1, grid, dx, deta, dtau, eos, eta_over_s, zeta_over_s, opt);
}

int kt_set_state_event(kt_ctx* c, int event, double tau, const double* e, const double* u, const double* pi,
                       const double* Pi, const double* u_prev, int on_device) {
  Range range_("kt_set_state");
  if (!c) return KT_ERR_ARG;
  if (event < 0 || event >= c->nev || !e || !(tau > 0 || !c->P.milne))
    return fail(c, KT_ERR_ARG, "kt_set_state: bad argument");
  const Lattice& L = c->lat[event];
  size_t ncp = (size_t)L.nx * L.ny * L.nz;
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  double* s = c->stage;
  CK(cudaMemcpyAsync(s, e, ncp * 8, kind, c->stream));
  if (u) CK(cudaMemcpyAsync(s + ncp, u, 3 * ncp * 8, kind, c->stream));
  if (pi) CK(cudaMemcpyAsync(s + 4 * ncp, pi, 10 * ncp * 8, kind, c->stream));
  if (Pi) CK(cudaMemcpyAsync(s + 14 * ncp, Pi, ncp * 8, kind, c->stream));
  if (u_prev) CK(cudaMemcpyAsync(s + 15 * ncp, u_prev, 3 * ncp * 8, kind, c->stream));
  CK(cudaMemsetAsync(c->d_stat, 0, 256, c->stream));
  double tau_h = tau;
  CK(cudaMemcpyAsync(c->d_tau, &tau_h, 8, cudaMemcpyHostToDevice, c->stream));
  int nb = (int)((ncp + 255) / 256);
  // the state goes into the buffers that hold u^n and u^{n-1} in the current rotation
  if (c->mixed)
    set_state_kernel<float><<<nb, 256, 0, c->stream>>>(c->P, L, s, u != nullptr, pi != nullptr, Pi != nullptr,
                                                       u_prev != nullptr, tau, c->q, c->qf, (float*)c->U[c->cur],
                                                       (float*)c->U[c->prev], (float*)c->E[0], (float*)c->Pb[0],
                                                       c->reg, c->d_stat);
  else
    set_state_kernel<double><<<nb, 256, 0, c->stream>>>(c->P, L, s, u != nullptr, pi != nullptr, Pi != nullptr,
                                                        u_prev != nullptr, tau, c->q, nullptr, (double*)c->U[c->cur],
                                                        (double*)c->U[c->prev], (double*)c->E[0], (double*)c->Pb[0],
                                                        c->reg, c->d_stat);
  CK(cudaGetLastError());
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, c->d_stat, 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->tau = tau;
  c->steps = 0;
  c->ev_set[event] = 1;
  if (st & ST_NONFINITE) return fail(c, KT_ERR_STATE, "kt_set_state: non-finite input or negative e");
  if (st) return fail(c, KT_ERR_STATE, "kt_set_state: T^{tau tau} - pi^{tau tau} <= |T^{tau i} - pi^{tau i}| "
                                       "in some cell (no (e, u) solves Eq. eInferred)");
  return KT_OK;
}

int kt_set_state(kt_ctx* c, double tau, const double* e, const double* u, const double* pi, const double* Pi,
                 const double* u_prev, int on_device) {
  return kt_set_state_event(c, 0, tau, e, u, pi, Pi, u_prev, on_device);
}

}  // extern "C"

namespace {

int begin_steps(Ctx* c, int n_steps) {
  for (int e = 0; e < c->nev; ++e)
    if (!c->ev_set[e]) return fail(c, KT_ERR_ARG, "kt_step: event %d has no state", e);
  if (c->opt.autotune && !c->tuned && n_steps > 0) {
    int rc = autotune(c);
    if (rc != KT_OK) return rc;
  }
  CK(cudaMemsetAsync(c->d_stat, 0, 256, c->stream));
  return KT_OK;
}

// read the statistics of the steps just enqueued (one synchronisation) and advance the host tau
int finish_steps(Ctx* c, int n_steps) {
  unsigned hst[KSTAT_WORDS];
  CK(cudaMemcpyAsync(hst, c->d_stat, sizeof(hst), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int s = 0; s < n_steps; ++s) c->tau += c->P.dtau;
  c->steps += n_steps;
  unsigned long long cnt[3];
  memcpy(cnt, &hst[4], sizeof(cnt));
  c->last.status = hst[0];
  float ms;
  memcpy(&ms, &hst[1], 4);
  c->last.max_speed = ms;
  c->last.newton_iters = (long long)cnt[0];
  c->last.regulated = (long long)cnt[1];
  c->last.fallbacks = (long long)cnt[2];
  if (hst[0] & ST_TIMEOUT) return fail(c, KT_ERR_TIMEOUT, "kt_step: a shared-memory copy timed out");
  if (hst[0] & ST_NONFINITE) return fail(c, KT_ERR_NONFINITE, "kt_step: non-finite value");
  if (hst[0] & ST_INVERSION) return fail(c, KT_ERR_INVERSION, "kt_step: inversion failed in some cell");
  return KT_OK;
}

}  // namespace

extern "C" {

int kt_step(kt_ctx* c, int n_steps) {
  Range range_("kt_step");
  if (!c || n_steps < 0) return KT_ERR_ARG;
  int rc = begin_steps(c, n_steps);
  if (rc != KT_OK) return rc;
  int done = 0;
  if (c->opt.use_graph) {
    while (n_steps - done >= 3) {
      int ph = c->cur;  // the three rotation phases are told apart by the current u buffer
      if (!c->graph[ph]) {
        rc = build_graph(c, ph);
        if (rc != KT_OK) return rc;
      }
      CK(cudaGraphLaunch(c->graph[ph], c->stream));
      done += 3;  // three steps return the rotation to the same phase
    }
  }
  for (; done < n_steps; ++done) {
    rc = enqueue_step(c);
    if (rc != KT_OK) return rc;
  }
  return finish_steps(c, n_steps);
}

int kt_time_kernels(kt_ctx* c, int n_steps, float* ms, int* n_kernels) {
  Range range_("kt_time_kernels");
  if (!c || n_steps < 1 || !ms || !n_kernels || *n_kernels < kNumTimed) return KT_ERR_ARG;
  int rc = begin_steps(c, n_steps);
  if (rc != KT_OK) return rc;
  cudaEvent_t ev[kNumTimed + 1];
  for (int k = 0; k <= kNumTimed; ++k) CK(cudaEventCreate(&ev[k]));
  double acc[kNumTimed] = {0.0};
  for (int s = 0; s < n_steps && rc == KT_OK; ++s) {
    rc = enqueue_step(c, ev);
    if (rc != KT_OK) break;
    cudaError_t e = cudaEventSynchronize(ev[kNumTimed]);
    if (e != cudaSuccess) { rc = fail(c, KT_ERR_CUDA, "kt_time_kernels: %s", cudaGetErrorString(e)); break; }
    for (int k = 0; k < kNumTimed; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
  }
  for (int k = 0; k <= kNumTimed; ++k) cudaEventDestroy(ev[k]);
  if (rc != KT_OK) return rc;
  for (int k = 0; k < kNumTimed; ++k) ms[k] = (float)(acc[k] / n_steps);
  *n_kernels = kNumTimed;
  return finish_steps(c, n_steps);
}

int kt_get_state_event(kt_ctx* c, int event, double* tau, double* e, double* u, double* pi, double* Pi, double* q,
                       int on_device) {
  Range range_("kt_get_state");
  if (!c) return KT_ERR_ARG;
  if (event < 0 || event >= c->nev) return fail(c, KT_ERR_ARG, "kt_get_state: bad event");
  const Lattice& L = c->lat[event];
  size_t ncp = (size_t)L.nx * L.ny * L.nz;
  const long long fs = c->gs;
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int nb = (int)((ncp + 255) / 256);
  // (source component, destination) pairs, gathered through the staging area in groups
  struct Job { const void* f; int is_r; double* dst; };
  std::vector<Job> jobs;
  const char* Ucur = (const char*)c->U[c->cur];
  if (e) jobs.push_back({c->E[0], 1, e});
  if (u) for (int m = 0; m < 4; ++m) jobs.push_back({Ucur + (size_t)m * fs * c->esz, 1, u + m * ncp});
  // component n of q: FP64, or (KT_STORE_PI_FP32, n >= 4) the FP32 state
  auto qjob = [&](int n, double* dst) {
    if (c->pi32 && n >= 4) jobs.push_back({c->qf + (size_t)n * fs, 2, dst});
    else jobs.push_back({c->q + (size_t)n * fs, 0, dst});
  };
  if (pi) for (int m = 0; m < 10; ++m) qjob(4 + m, pi + m * ncp);
  if (Pi) qjob(14, Pi);
  if (q) for (int n = 0; n < NQ; ++n) qjob(n, q + n * ncp);
  for (size_t b = 0; b < jobs.size(); b += 18) {
    size_t nj = std::min<size_t>(18, jobs.size() - b);
    for (size_t t = 0; t < nj; ++t) {
      const Job& jb = jobs[b + t];
      double* dst = c->stage + t * ncp;
      if (jb.is_r == 2 || (jb.is_r && c->mixed))
        gather_kernel<float><<<nb, 256, 0, c->stream>>>(L, (const float*)jb.f, dst);
      else gather_kernel<double><<<nb, 256, 0, c->stream>>>(L, (const double*)jb.f, dst);
    }
    CK(cudaGetLastError());
    for (size_t t = 0; t < nj; ++t) CK(cudaMemcpyAsync(jobs[b + t].dst, c->stage + t * ncp, ncp * 8, kind, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  if (tau) *tau = c->tau;
  return KT_OK;
}

int kt_get_state(kt_ctx* c, double* tau, double* e, double* u, double* pi, double* Pi, double* q, int on_device) {
  return kt_get_state_event(c, 0, tau, e, u, pi, Pi, q, on_device);
}

}  // extern "C"

namespace {

// The fields of a checkpoint row by row (see KT_CHECKPOINT_ROWS in kt.h): the field array (all
// events) and its element type: 0 double, 1 the stencil precision (float in KT_MIXED), 2 float.
struct CkptRow {
  void* f;
  int is_r;
};
std::vector<CkptRow> checkpoint_rows(Ctx* c) {
  std::vector<CkptRow> rows;
  const size_t fs = (size_t)c->gs;
  for (int n = 0; n < NQ; ++n)
    rows.push_back((c->pi32 && n >= 4) ? CkptRow{c->qf + n * fs, 2} : CkptRow{c->q + n * fs, 0});
  for (int n = 0; n < NQ; ++n)
    rows.push_back(c->mixed ? CkptRow{c->qf + n * fs, 1} : CkptRow{c->q + n * fs, 0});
  rows.push_back({c->E[0], 1});
  rows.push_back({c->Pb[0], 1});
  for (int m = 0; m < 4; ++m) rows.push_back({(char*)c->U[c->cur] + m * fs * c->esz, 1});
  for (int m = 0; m < 4; ++m) rows.push_back({(char*)c->U[c->prev] + m * fs * c->esz, 1});
  rows.push_back({c->reg, 2});  // float in both modes
  return rows;
}

}  // namespace

extern "C" {

int kt_get_checkpoint(kt_ctx* c, int event, double* tau, double* buf, int on_device) {
  Range range_("kt_get_checkpoint");
  if (!c || !buf) return KT_ERR_ARG;
  if (event < 0 || event >= c->nev) return fail(c, KT_ERR_ARG, "kt_get_checkpoint: bad event");
  if (!c->ev_set[event]) return fail(c, KT_ERR_ARG, "kt_get_checkpoint: event %d has no state", event);
  const Lattice& L = c->lat[event];
  const size_t ncp = (size_t)L.nx * L.ny * L.nz;
  const int nb = (int)((ncp + 255) / 256);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const std::vector<CkptRow> rows = checkpoint_rows(c);
  static_assert(KT_CHECKPOINT_ROWS == 41, "checkpoint layout");
  for (size_t b = 0; b < rows.size(); b += 18) {  // through the staging area, 18 rows at a time
    const size_t nr = std::min<size_t>(18, rows.size() - b);
    for (size_t t = 0; t < nr; ++t) {
      const CkptRow& r = rows[b + t];
      double* dst = c->stage + t * ncp;
      if (r.is_r == 2 || (r.is_r && c->mixed)) gather_kernel<float><<<nb, 256, 0, c->stream>>>(L, (const float*)r.f, dst);
      else gather_kernel<double><<<nb, 256, 0, c->stream>>>(L, (const double*)r.f, dst);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(buf + b * ncp, c->stage, nr * ncp * 8, kind, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  if (tau) *tau = c->tau;
  return KT_OK;
}

int kt_set_checkpoint(kt_ctx* c, int event, double tau, const double* buf, int on_device) {
  Range range_("kt_set_checkpoint");
  if (!c || !buf) return KT_ERR_ARG;
  if (event < 0 || event >= c->nev || !(tau > 0 || !c->P.milne))
    return fail(c, KT_ERR_ARG, "kt_set_checkpoint: bad argument");
  const Lattice& L = c->lat[event];
  const size_t ncp = (size_t)L.nx * L.ny * L.nz;
  const int nb = (int)((ncp + 255) / 256);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const std::vector<CkptRow> rows = checkpoint_rows(c);
  for (size_t b = 0; b < rows.size(); b += 18) {
    const size_t nr = std::min<size_t>(18, rows.size() - b);
    CK(cudaMemcpyAsync(c->stage, buf + b * ncp, nr * ncp * 8, kind, c->stream));
    for (size_t t = 0; t < nr; ++t) {
      const CkptRow& r = rows[b + t];
      const size_t row = b + t;
      if (!c->mixed && row >= (size_t)NQ && row < (size_t)(2 * NQ)) continue;  // FP64: the stencil reads q
      if (c->pi32 && row >= (size_t)(NQ + 4) && row < (size_t)(2 * NQ)) continue;  // the state rows hold them
      const double* src = c->stage + t * ncp;
      if (r.is_r == 2 || (r.is_r && c->mixed)) scatter_kernel<float><<<nb, 256, 0, c->stream>>>(c->P, L, src, (float*)r.f);
      else scatter_kernel<double><<<nb, 256, 0, c->stream>>>(c->P, L, src, (double*)r.f);
    }
    CK(cudaGetLastError());
  }
  double tau_h = tau;
  CK(cudaMemcpyAsync(c->d_tau, &tau_h, 8, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->d_stat, 0, 256, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->tau = tau;
  c->steps = 0;
  c->ev_set[event] = 1;
  return KT_OK;
}

int kt_selftest_wait(kt_ctx* c, unsigned polls) {
  if (!c || polls == 0) return KT_ERR_ARG;
  CK(cudaMemsetAsync(c->d_stat, 0, 4, c->stream));
  wait_selftest_kernel<<<1, 128, 0, c->stream>>>(polls, c->d_stat);
  CK(cudaGetLastError());
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, c->d_stat, 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st & ST_TIMEOUT) return fail(c, KT_ERR_TIMEOUT, "kt_selftest_wait: the wait gave up after %u polls", polls);
  return KT_OK;
}

int kt_selftest_cvt(const double* x, float* rn, float* rz, long long n, void* stream) {
  if (!x || !rn || !rz || n < 0) return KT_ERR_ARG;
  if (n == 0) return KT_OK;
  cvt_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, rn, rz, n);
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ERR_CUDA;
}

int kt_selftest_div(const double* a, const double* b, double* q, long long n, void* stream) {
  if (!a || !b || !q || n < 0) return KT_ERR_ARG;
  if (n == 0) return KT_OK;
  div_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a, b, q, n);
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ERR_CUDA;
}

int kt_get_diagnostics(kt_ctx* c, int event, double* out, int on_device) {
  Range range_("kt_get_diagnostics");
  if (!c || !out) return KT_ERR_ARG;
  if (event < 0 || event >= c->nev) return fail(c, KT_ERR_ARG, "kt_get_diagnostics: bad event");
  if (!c->ev_set[event]) return fail(c, KT_ERR_ARG, "kt_get_diagnostics: event %d has no state", event);
  const Lattice& L = c->lat[event];
  const size_t ncp = (size_t)L.nx * L.ny * L.nz;
  const int nb = (int)((ncp + 255) / 256);
  if (c->mixed) {
    StageIO<float> io = make_io<float>(c, 1);
    diag_kernel<float><<<nb, 256, 0, c->stream>>>(c->P, L, io, c->tau, c->reg, c->stage);
  } else {
    StageIO<double> io = make_io<double>(c, 1);
    diag_kernel<double><<<nb, 256, 0, c->stream>>>(c->P, L, io, c->tau, c->reg, c->stage);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, c->stage, 7 * ncp * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return KT_OK;
}

int kt_mlp_features(kt_ctx* c, long long n, const long long* cells, float* x, float* y, double* e_exact) {
  if (!c || n < 0 || !cells || !x || !y || !e_exact)
    return c ? fail(c, KT_ERR_ARG, "kt_mlp_features: bad argument") : KT_ERR_ARG;
  if (!c->ev_set[0]) return fail(c, KT_ERR_ARG, "kt_mlp_features: no state set");
  if (n == 0) return KT_OK;
  CK(cudaMemsetAsync(c->d_stat, 0, 4, c->stream));
  mlp_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->P, c->lat[0], c->q, c->qf, c->pi32,
                                                                          c->tau, n, cells, x, y, e_exact, c->d_stat);
  CK(cudaGetLastError());
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, c->d_stat, 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st) return fail(c, KT_ERR_INVERSION, "kt_mlp_features: bad cell index or failed root-find");
  return KT_OK;
}

int kt_get_tuning(kt_ctx* c, int* block_xyz, int* grid_blocks, float* candidate_ms, int* n_candidates) {
  if (!c) return KT_ERR_ARG;
  if (block_xyz) {
    block_xyz[0] = kShapes[c->shape].x;
    block_xyz[1] = kShapes[c->shape].y;
    block_xyz[2] = kShapes[c->shape].z;
  }
  if (grid_blocks) *grid_blocks = c->grid_blocks;
  if (n_candidates) {
    if (candidate_ms)
      for (int s = 0; s < std::min(*n_candidates, kNumCandidates); ++s)
        candidate_ms[s] = c->tuned ? c->tune_ms[s] : 0.f;
    *n_candidates = kNumCandidates;
  }
  return KT_OK;
}

int kt_set_tuning(kt_ctx* c, int candidate) {
  if (!c || candidate < 0 || candidate >= kNumCandidates) return KT_ERR_ARG;
  int rc = select_shape(c, candidate);
  if (rc != KT_OK) return rc;
  c->tuned = true;  // no autotuning on the next step
  return KT_OK;
}

int kt_get_stats(kt_ctx* c, kt_stats* s) {
  if (!c || !s) return KT_ERR_ARG;
  kt_stats r = c->last;
  r.tau = c->tau;
  r.steps = c->steps;
  r.e_min = r.e_max = r.reg_min = 0.0;
  bool any = false;
  for (int e = 0; e < c->nev; ++e) any |= (c->ev_set[e] != 0);
  if (any) {  // the extrema of the current state, reduced on the device (words 12-14 of the stats block)
    unsigned* ext = c->d_stat + KSTAT_WORDS;
    const unsigned init[3] = {0x7f800000u, 0u, 0x7f800000u};
    CK(cudaMemcpyAsync(ext, init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
    for (int e = 0; e < c->nev; ++e) {
      if (!c->ev_set[e]) continue;
      if (c->mixed) state_extrema_kernel<float><<<152, 256, 0, c->stream>>>(c->lat[e], (const float*)c->E[0], c->reg, ext);
      else state_extrema_kernel<double><<<152, 256, 0, c->stream>>>(c->lat[e], (const double*)c->E[0], c->reg, ext);
    }
    CK(cudaGetLastError());
    unsigned h[3];
    CK(cudaMemcpyAsync(h, ext, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    float f[3];
    memcpy(f, h, sizeof(f));
    r.e_min = f[0];
    r.e_max = f[1];
    r.reg_min = f[2];
  }
  *s = r;
  return KT_OK;
}

const char* kt_last_error(const kt_ctx* c) { return c ? c->err : "null context"; }

void kt_free(kt_ctx* c) {
  if (!c) return;
  for (int p = 0; p < 3; ++p)
    if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
  if (c->base) cudaFree(c->base);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
