// kt_mlp.cu -- training and stand-alone inference kernels of the learned root-find start.
//
// Training (SIMT, FP32 accumulation): the forward pass rounds weights and activations to
// BF16 exactly as the tensor-core inference does (bf16_forward = 1), or runs in plain FP32
// (bf16_forward = 0, used to check gradients against the FP64 reference); the backward pass
// treats the rounding as the identity.  Gradients of a mini-batch are reduced with warp
// shuffles, then shared-memory and global atomics.  Adam updates FP32 master weights.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/kt.h"
#include "kt_mlp.cuh"

using namespace kt;

// Scratch of kt_mlp_predict_static: one packed weight set, KT_MLP_PACKED_BYTES bytes, in a
// file-scope device array.  Every GPU that loads this library holds it until the process
// exits.  In host code `g_predict_scratch` is only a host-side stand-in for the symbol: its
// device address comes from cudaGetSymbolAddress, looked up once per device and context and
// cached below.  The cache is keyed on the context's unique id as well as the device, so a
// context re-created on the same device (after cudaDeviceReset, whose new module instance may
// hold the array elsewhere) gets a fresh lookup instead of a stale address.
static __device__ __align__(256) uint32_t g_predict_scratch[kt::PK_WORDS];

namespace {
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  unsigned long long ctx_id;
  uint32_t* ptr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// the unique id of the calling thread's current context (0 if there is none yet or the driver
// entry points are unavailable)
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)f;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// device address of g_predict_scratch on the current device and context (looked up on the first
// call there; cudaGetSymbolAddress allocates nothing)
int static_scratch_address(uint32_t** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return KT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return KT_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  const unsigned long long id = current_context_id();
  ScratchAddr& a = g_scratch_addr[dev];
  if (!a.ptr || id == 0 || a.ctx_id != id) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_predict_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "kt_mlp_predict_static: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return KT_ERR_CUDA;
    }
    a.ptr = (uint32_t*)p;
    a.ctx_id = current_context_id();  // the lookup has made the device's context current
  }
  *out = a.ptr;
  return KT_OK;
}
}  // namespace

namespace {

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool BF16>
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float* __restrict__ params, const float* __restrict__ X,
                                                       const float* __restrict__ Y, long long n, float inv_n,
                                                       float* grad, float* loss) {
  __shared__ float sw[MLP_NPARAM];
  __shared__ float sg[MLP_NPARAM];
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x) {
    sw[p] = BF16 ? bf16r(params[p]) : params[p];
    sg[p] = 0.f;
  }
  // biases are applied in FP32 by the tensor-core path too
  for (int p = threadIdx.x; p < MLP_H; p += blockDim.x) {
    sw[OFF_B1 + p] = params[OFF_B1 + p];
    sw[OFF_B2 + p] = params[OFF_B2 + p];
  }
  if (threadIdx.x == 0) sw[OFF_B3] = params[OFF_B3];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  float x[MLP_IN];
#pragma unroll
  for (int k = 0; k < MLP_IN; ++k) x[k] = valid ? (BF16 ? bf16r(X[i * MLP_IN + k]) : X[i * MLP_IN + k]) : 0.f;
  const float yt = valid ? Y[i] : 0.f;
  // forward
  float h1[MLP_H], h2[MLP_H];
#pragma unroll 4
  for (int j = 0; j < MLP_H; ++j) {
    float s = sw[OFF_B1 + j];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) s += sw[OFF_W1 + j * MLP_IN + k] * x[k];
    s = fmaxf(s, 0.f);
    h1[j] = BF16 ? bf16r(s) : s;
  }
#pragma unroll 2
  for (int j = 0; j < MLP_H; ++j) {
    float s = sw[OFF_B2 + j];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) s += sw[OFF_W2 + j * MLP_H + k] * h1[k];
    s = fmaxf(s, 0.f);
    h2[j] = BF16 ? bf16r(s) : s;
  }
  float y = sw[OFF_B3];
#pragma unroll
  for (int k = 0; k < MLP_H; ++k) y += sw[OFF_W3 + k] * h2[k];
  // mean squared error
  const float r = valid ? (y - yt) : 0.f;
  const float dy = 2.f * r * inv_n;
  const float lsum = warp_sum(r * r * inv_n);
  const int lane = threadIdx.x & 31;
  if (lane == 0) atomicAdd(loss, lsum);
  // backward, each parameter's contribution summed over the warp
  {
    float s = warp_sum(dy);
    if (lane == 0) atomicAdd(&sg[OFF_B3], s);
  }
  float d2[MLP_H];
#pragma unroll 1
  for (int k = 0; k < MLP_H; ++k) {
    float s = warp_sum(dy * h2[k]);
    if (lane == 0) atomicAdd(&sg[OFF_W3 + k], s);
  }
#pragma unroll
  for (int k = 0; k < MLP_H; ++k) d2[k] = (h2[k] > 0.f) ? dy * sw[OFF_W3 + k] : 0.f;
#pragma unroll 1
  for (int j = 0; j < MLP_H; ++j) {
    float s = warp_sum(d2[j]);
    if (lane == 0) atomicAdd(&sg[OFF_B2 + j], s);
#pragma unroll 1
    for (int k = 0; k < MLP_H; ++k) {
      float t = warp_sum(d2[j] * h1[k]);
      if (lane == 0) atomicAdd(&sg[OFF_W2 + j * MLP_H + k], t);
    }
  }
  float d1[MLP_H];
#pragma unroll 1
  for (int k = 0; k < MLP_H; ++k) {
    float s = 0.f;
#pragma unroll 8
    for (int j = 0; j < MLP_H; ++j) s += d2[j] * sw[OFF_W2 + j * MLP_H + k];
    d1[k] = (h1[k] > 0.f) ? s : 0.f;
  }
#pragma unroll 1
  for (int j = 0; j < MLP_H; ++j) {
    float s = warp_sum(d1[j]);
    if (lane == 0) atomicAdd(&sg[OFF_B1 + j], s);
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) {
      float t = warp_sum(d1[j] * x[k]);
      if (lane == 0) atomicAdd(&sg[OFF_W1 + j * MLP_IN + k], t);
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x) atomicAdd(&grad[p], sg[p]);
}

__global__ void mlp_adam_kernel(float* params, const float* __restrict__ grad, float* m, float* v, float lr,
                                float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gp = grad[p];
  const float mp = b1 * m[p] + (1.f - b1) * gp;
  const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  params[p] -= lr * (mp * c1) / (sqrtf(vp * c2) + eps);
}

// ---------------------------------------------------------------- training data
// The training set keeps the samples the network corrects (feature 1, r^2 = M^2/E^2, above the
// gate) in their original order, with target z = y / r^2: a stable compaction in three passes
// (per-block counts, one-block scan of the counts, per-block scatter) over tiles of
// kTgtTile samples.
constexpr int kTgtThreads = 256, kTgtPer = 4, kTgtTile = kTgtThreads * kTgtPer;

__device__ __forceinline__ bool network_corrects(const float* __restrict__ x, long long i) {
  return x[i * MLP_IN + 1] > kMlpGateR2;
}

__global__ void __launch_bounds__(kTgtThreads) targets_count_kernel(const float* __restrict__ x, long long n,
                                                                    long long* counts) {
  __shared__ int s_w[kTgtThreads / 32];
  int c = 0;
  const long long base = (long long)blockIdx.x * kTgtTile;
#pragma unroll
  for (int k = 0; k < kTgtPer; ++k) {
    const long long i = base + k * kTgtThreads + threadIdx.x;
    c += (i < n && network_corrects(x, i)) ? 1 : 0;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kTgtThreads / 32; ++w) t += s_w[w];
    counts[blockIdx.x] = t;
  }
}

// exclusive scan of the per-block counts in place, total into *n_out (one block)
__global__ void __launch_bounds__(1024) targets_scan_kernel(long long* counts, long long nblocks, long long* n_out) {
  __shared__ long long s_part[1024];
  const long long per = (nblocks + blockDim.x - 1) / blockDim.x;
  const long long b0 = threadIdx.x * per, b1 = min(nblocks, b0 + per);
  long long t = 0;
  for (long long b = b0; b < b1; ++b) t += counts[b];
  s_part[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      const long long v = s_part[k];
      s_part[k] = acc;
      acc += v;
    }
    *n_out = acc;
  }
  __syncthreads();
  long long acc = s_part[threadIdx.x];
  for (long long b = b0; b < b1; ++b) {
    const long long v = counts[b];
    counts[b] = acc;
    acc += v;
  }
}

__global__ void __launch_bounds__(kTgtThreads) targets_scatter_kernel(const float* __restrict__ x,
                                                                      const float* __restrict__ y, long long n,
                                                                      const long long* __restrict__ offsets,
                                                                      float* x_out, float* z_out) {
  __shared__ int s_w[kTgtThreads / 32];
  long long off = offsets[blockIdx.x];
  const long long base = (long long)blockIdx.x * kTgtTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < kTgtPer; ++k) {  // samples in order: row k of the tile, then the threads
    const long long i = base + k * kTgtThreads + threadIdx.x;
    const bool keep = i < n && network_corrects(x, i);
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kTgtThreads / 32; ++w) {
      const int c = s_w[w];
      before += (w < warp) ? c : 0;
      total += c;
    }
    if (keep) {
      const long long o = off + before + __popc(bal & ((1u << lane) - 1u));
      const float r2 = x[i * MLP_IN + 1];
#pragma unroll
      for (int m = 0; m < MLP_IN; ++m) x_out[o * MLP_IN + m] = x[i * MLP_IN + m];
      z_out[o] = __fdiv_rn(y[i], r2);
    }
    off += total;
    __syncthreads();
  }
}

// A keyed pseudo-random permutation of [0, n): a 4-round balanced Feistel network on 2h-bit
// words (4^h >= n) with a SplitMix64-finalised round function, and cycle walking back into
// [0, n).  Each walk is bounded; a walk that has not returned after kWalkMax rounds (not expected:
// at most 3/4 of the domain lies outside [0, n)) takes i itself and is flagged.
constexpr int kWalkMax = 4096;
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long feistel(unsigned long long v, int h, unsigned long long key) {
  const unsigned long long mask = (1ULL << h) - 1ULL;
  unsigned long long L = v >> h, R = v & mask;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const unsigned long long F = mix64(R ^ (key + 0x9e3779b97f4a7c15ULL * (unsigned long long)(r + 1))) & mask;
    const unsigned long long t = L ^ F;
    L = R;
    R = t;
  }
  return (L << h) | R;
}

__global__ void batch_kernel(const float* __restrict__ x, const float* __restrict__ y, long long n, int h,
                             unsigned long long key, long long first, long long count, float* xb, float* yb,
                             unsigned* flag) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  unsigned long long v = (unsigned long long)(first + k);
  int w = 0;
  do {
    v = feistel(v, h, key);
  } while (v >= (unsigned long long)n && ++w < kWalkMax);
  if (v >= (unsigned long long)n) {
    v = (unsigned long long)(first + k);
    atomicOr(flag, 1u);
  }
#pragma unroll
  for (int m = 0; m < MLP_IN; ++m) xb[k * MLP_IN + m] = x[v * MLP_IN + m];
  yb[k] = y[v];
}

}  // namespace

namespace kt {
// FP32 parameters -> packed BF16 fragments + FP32 biases (see kt_mlp.cuh)
__global__ void mlp_pack_kernel(const float* __restrict__ params, uint32_t* packed) {
  for (int i = threadIdx.x; i < PK_WORDS; i += blockDim.x) {
    uint32_t v = 0u;
    if (i < PK_W2) {  // W1 rows of 4 words
      const int n = i / 4, w = i % 4, k = 2 * w;
      const float lo = (k < MLP_IN) ? params[OFF_W1 + n * MLP_IN + k] : 0.f;
      const float hi = (k + 1 < MLP_IN) ? params[OFF_W1 + n * MLP_IN + k + 1] : 0.f;
      v = pack_bf16x2(lo, hi);
    } else if (i < PK_W3) {  // W2 rows of 20 words (16 used)
      const int n = (i - PK_W2) / PK_W2_STRIDE, w = (i - PK_W2) % PK_W2_STRIDE;
      if (w < 16) v = pack_bf16x2(params[OFF_W2 + n * MLP_H + 2 * w], params[OFF_W2 + n * MLP_H + 2 * w + 1]);
    } else if (i < PK_B1) {
      const int w = i - PK_W3;
      v = pack_bf16x2(params[OFF_W3 + 2 * w], params[OFF_W3 + 2 * w + 1]);
    } else if (i < PK_B2) {
      v = __float_as_uint(params[OFF_B1 + (i - PK_B1)]);
    } else if (i < PK_B3) {
      v = __float_as_uint(params[OFF_B2 + (i - PK_B2)]);
    } else {
      v = __float_as_uint(params[OFF_B3]);
    }
    packed[i] = v;
  }
}

// tensor-core inference over an array of feature rows
__global__ void __launch_bounds__(256) mlp_predict_kernel(const uint32_t* __restrict__ packed,
                                                          const float* __restrict__ X, long long n, float* Y) {
  __shared__ alignas(16) uint32_t sw[PK_WORDS];
  mlp_load_shared(sw, packed);
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float x[MLP_IN];
#pragma unroll
  for (int k = 0; k < MLP_IN; ++k) x[k] = (i < n) ? X[i * MLP_IN + k] : 0.f;
  const float y = mlp_warp_infer(sw, x);  // every lane of the warp takes part
  if (i < n) Y[i] = y;
}
}  // namespace kt

extern "C" {

int kt_mlp_predict(const float* params, const float* x, long long n, float* y, void* scratch, size_t scratch_bytes,
                   void* stream) {
  if (!params || !x || !y || n < 0 || !scratch || scratch_bytes < (size_t)KT_MLP_PACKED_BYTES) return KT_ERR_ARG;
  if (n == 0) return KT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  kt::mlp_pack_kernel<<<1, 256, 0, s>>>(params, (uint32_t*)scratch);
  kt::mlp_predict_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const uint32_t*)scratch, x, n, y);
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ERR_CUDA;
}

int kt_mlp_predict_static(const float* params, const float* x, long long n, float* y, void* stream) {
  if (!params || !x || !y || n < 0) {
    fprintf(stderr, "kt_mlp_predict_static: null pointer or negative row count\n");
    return KT_ERR_ARG;
  }
  if (n > KT_MLP_STATIC_MAX_ROWS) {
    fprintf(stderr, "kt_mlp_predict_static: %lld rows exceed the maximum of %lld\n", n,
            (long long)KT_MLP_STATIC_MAX_ROWS);
    return KT_ERR_ARG;
  }
  if (n == 0) return KT_OK;
  uint32_t* scratch = nullptr;
  const int rc = static_scratch_address(&scratch);
  if (rc != KT_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // the pack kernel overwrites every word of the scratch, so nothing needs clearing first
  kt::mlp_pack_kernel<<<1, 256, 0, s>>>(params, scratch);
  kt::mlp_predict_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(scratch, x, n, y);
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ERR_CUDA;
}

int kt_mlp_grad(const float* params, const float* x, const float* y_target, long long n, int bf16_forward,
                float* grad, float* loss, void* stream) {
  if (!params || !x || !y_target || !grad || !loss || n <= 0) return KT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(grad, 0, KT_MLP_NPARAM * sizeof(float), s) != cudaSuccess) return KT_ERR_CUDA;
  if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return KT_ERR_CUDA;
  const unsigned nb = (unsigned)((n + 255) / 256);
  const float inv_n = (float)(1.0 / (double)n);
  if (bf16_forward)
    mlp_grad_kernel<true><<<nb, 256, 0, s>>>(params, x, y_target, n, inv_n, grad, loss);
  else
    mlp_grad_kernel<false><<<nb, 256, 0, s>>>(params, x, y_target, n, inv_n, grad, loss);
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ERR_CUDA;
}

int kt_mlp_targets_workspace(long long n, size_t* bytes) {
  if (n < 0 || !bytes) return KT_ERR_ARG;
  *bytes = (size_t)((n + kTgtTile - 1) / kTgtTile + 1) * sizeof(long long);
  return KT_OK;
}

int kt_mlp_targets(const float* x, const float* y, long long n, float* x_out, float* z_out, long long* n_out,
                   void* workspace, size_t workspace_bytes, void* stream) {
  size_t need = 0;
  if (!x || !y || !x_out || !z_out || !n_out || !workspace || kt_mlp_targets_workspace(n, &need) != KT_OK ||
      workspace_bytes < need)
    return KT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long nb = (n + kTgtTile - 1) / kTgtTile;
  long long* counts = (long long*)workspace;
  if (nb == 0) return cudaMemsetAsync(n_out, 0, sizeof(long long), s) == cudaSuccess ? KT_OK : KT_ERR_CUDA;
  if (nb > 0x7fffffffLL) return KT_ERR_ARG;
  targets_count_kernel<<<(unsigned)nb, kTgtThreads, 0, s>>>(x, n, counts);
  targets_scan_kernel<<<1, 1024, 0, s>>>(counts, nb, n_out);
  targets_scatter_kernel<<<(unsigned)nb, kTgtThreads, 0, s>>>(x, y, n, counts, x_out, z_out);
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ERR_CUDA;
}

int kt_mlp_batch(const float* x, const float* y, long long n, unsigned long long seed, int epoch, long long b,
                 long long batch, float* xb, float* yb, unsigned* flag, void* stream) {
  if (!x || !y || !xb || !yb || !flag || n <= 0 || batch <= 0 || b < 0 || epoch < 0) return KT_ERR_ARG;
  const long long first = b * batch;
  if (first >= n) return KT_ERR_ARG;
  const long long count = (first + batch <= n) ? batch : n - first;
  int h = 1;
  while (h < 31 && (1LL << (2 * h)) < n) ++h;
  const unsigned long long key = seed * 0x2545f4914f6cdd1dULL + (unsigned long long)epoch;
  batch_kernel<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n, h, key, first, count, xb,
                                                                                    yb, flag);
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ERR_CUDA;
}

int kt_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream) {
  if (!params || !grad || !m || !v || step < 1 || !(lr > 0.f)) return KT_ERR_ARG;
  const double c1 = 1.0 / (1.0 - std::pow(0.9, step)), c2 = 1.0 / (1.0 - std::pow(0.999, step));
  mlp_adam_kernel<<<(KT_MLP_NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, lr, (float)c1,
                                                                                 (float)c2);
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ERR_CUDA;
}

}  // extern "C"
