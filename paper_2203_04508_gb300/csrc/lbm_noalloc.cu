// Mass audit that allocates nothing: a variant of the library's FP64 mass reduction whose
// scratch (per-block partial sums, the last-block counter and the result) lives in a
// file-scope device array instead of a caller workspace.
//
// Who needs it: code that must not call cudaMalloc, directly or through an allocator -- for
// example a host callback, a signal-safe monitor, or a process that has handed its whole
// device-memory budget to another framework's pool -- but already holds the populations it
// wants audited in device memory.  Such a caller passes its inputs and one host output and
// nothing is allocated on its behalf.
//
// The array is shared by every call in the process and keeps the last call's contents; each
// call clears the counter it relies on before launching.  Two calls whose kernels overlap on
// the GPU (different streams, or different host threads) race on it and must be serialised
// by the caller.
#include <cstdio>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_MAX_BLOCKS = 1024;
// layout of the scratch array, in doubles:
//   [0]           last-block counter (as unsigned int in the first 4 bytes)
//   [8], [9]      result: mass, non-finite count
//   [32 ...)      2 * NA_MAX_BLOCKS per-block partials
constexpr int NA_RESULT = 8;
constexpr int NA_PARTIALS = 32;
constexpr int NA_DOUBLES = NA_PARTIALS + 2 * NA_MAX_BLOCKS;   // 16,640 bytes

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

__device__ __forceinline__ double na_block_sum(double v, double* smem) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? smem[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// sum over nodes with kind == 0 of the 9 planes of f, in FP64, deterministic order
template <typename real>
__global__ void __launch_bounds__(NA_BLOCK) k_mass_noalloc(const real* __restrict__ f,
                                                           const uint8_t* __restrict__ kind, long long n,
                                                           double* scratch) {
  __shared__ double red[32];
  __shared__ double red2[32];
  __shared__ bool last;
  double s = 0.0, bad = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    if (kind[k] != 0) continue;
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      real v = f[i * n + k];
      if (!isfinite(v)) bad += 1.0;
      t += (double)v;
    }
    s += t;
  }
  const double bs = na_block_sum(s, red);
  const double bb = na_block_sum(bad, red2);
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
  double* partials = scratch + NA_PARTIALS;
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bs;
    partials[2 * blockIdx.x + 1] = bb;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, c = 0.0;
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
    a += ((volatile double*)partials)[2 * k];
    c += ((volatile double*)partials)[2 * k + 1];
  }
  const double ta = na_block_sum(a, red);
  const double tc = na_block_sum(c, red2);
  if (threadIdx.x == 0) {
    scratch[NA_RESULT] = ta;
    scratch[NA_RESULT + 1] = tc;
    *counter = 0u;
  }
}

// Device address of the scratch array in the current device's context.  It is looked up on
// every call rather than cached: a context that was torn down (cudaDeviceReset) and created
// again reloads the module, and an address kept from the old context would no longer be valid.
cudaError_t scratch_on_current_device(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_mass_noalloc(const void* f, const uint8_t* kind, int64_t n_nodes, int32_t precision,
                                       void* stream, double* out2) {
  if (!f || !kind || !out2) return LBM_EINVAL;
  if (n_nodes <= 0 || n_nodes > LBM_NOALLOC_MAX_NODES) {
    std::fprintf(stderr, "lbm_mass_noalloc: n_nodes=%lld outside [1, %lld]\n", (long long)n_nodes,
                 (long long)LBM_NOALLOC_MAX_NODES);
    return LBM_EINVAL;
  }
  if (precision != LBM_FP32 && precision != LBM_FP64) return LBM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the call ends in a pageable copy and a synchronisation, which a capture cannot hold
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return LBM_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return LBM_ESTATE;
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) return LBM_ECUDA;
  if (cudaMemsetAsync(scratch, 0, sizeof(double), s) != cudaSuccess) return LBM_ECUDA;   // the counter
  long long blocks = (n_nodes + NA_BLOCK - 1) / NA_BLOCK;
  if (blocks > NA_MAX_BLOCKS) blocks = NA_MAX_BLOCKS;
  if (precision == LBM_FP32)
    k_mass_noalloc<float><<<(unsigned)blocks, NA_BLOCK, 0, s>>>(static_cast<const float*>(f), kind, n_nodes, scratch);
  else
    k_mass_noalloc<double><<<(unsigned)blocks, NA_BLOCK, 0, s>>>(static_cast<const double*>(f), kind, n_nodes, scratch);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  if (cudaMemcpyAsync(out2, scratch + NA_RESULT, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return LBM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ECUDA;
  return LBM_OK;
}
