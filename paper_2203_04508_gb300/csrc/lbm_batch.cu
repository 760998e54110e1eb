// Batched persistent step: many independent lattices (of different sizes and physics) advanced
// together, n steps in one cooperative launch.
//
// Every phase of a step runs over a flat work list that spans all instances -- 2D tiles of 256
// nodes for the node phases, chunks of 256 entries for the solid-layer lists and
// the boundary nodes -- so that small and large lattices share the GPU evenly.  Between phases
// all blocks meet at a grid barrier (the blocks are co-resident: cooperative launch).  The
// barrier's wait is bounded: after `spin_limit` polls it sets an error flag and every block
// leaves the kernel, which the host reports as LBM_ETIMEOUT.
//
// The per-node arithmetic is that of the single-lattice kernels (lbm_phases.cuh); only the
// scheduling differs.
#include "lbm_internal.h"
#include "lbm_phases.cuh"

namespace lbmgb {

constexpr int BATCH_BLOCK = 256;

// Grid barrier.  bar[0] counts arrivals, bar[1] is the number of barriers completed in this
// launch (both zeroed before the launch); `target` is this barrier's ordinal (1, 2, ...).
__device__ __forceinline__ bool grid_sync(const BatchDev& B, unsigned int target) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned int arrived = atomicAdd(B.bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(B.bar, 0u);
      __threadfence();
      atomicExch(B.bar + 1, target);
    } else {
      volatile unsigned int* gen = B.bar + 1;
      volatile int* err = B.err;
      long long it = 0;
      while (*gen < target) {
        if (*err || ++it > B.spin_limit) {
          atomicExch(B.err, 1);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Copy of an instance's lattice descriptor into shared memory.  Each block takes a contiguous
// range of every work list, so consecutive items mostly belong to one instance and the copy
// is redone only when the instance changes.
template <typename real>
__device__ __forceinline__ void load_lattice(Lattice<real>& dst, const Lattice<real>* lat, int k, int& loaded) {
  if (k == loaded) return;   // block-uniform
  constexpr int W = (int)(sizeof(Lattice<real>) / sizeof(int));
  static_assert(sizeof(Lattice<real>) % sizeof(int) == 0, "descriptor size");
  __syncthreads();
  const int* s = reinterpret_cast<const int*>(lat + k);
  int* d = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < W; i += blockDim.x) d[i] = s[i];
  __syncthreads();
  loaded = k;
}

// this block's share [w0, w1) of a list of n items
__device__ __forceinline__ void block_range(int n, int& w0, int& w1) {
  w0 = (int)(((long long)n * blockIdx.x) / gridDim.x);
  w1 = (int)(((long long)n * (blockIdx.x + 1)) / gridDim.x);
}

// Node tiles are 2D blocks of 2^tile_log2w x (256 / 2^tile_log2w) nodes of an instance's
// lattice, row-major over the tiles of each instance: tile t of an instance with tiles_x tiles
// per row band covers x in [w (t % tiles_x), +w), y in [h (t / tiles_x), +h).  The shape is a
// run-time choice (lbm_batch_set_tile, lbm_batch_autotune); every shape gives the same values,
// since each node's arithmetic does not depend on it.  False outside the lattice.
template <typename real>
__device__ __forceinline__ bool tile_node(const Lattice<real>& L, int log2w, int t, int& x, int& y) {
  const int w = 1 << log2w, h = BATCH_BLOCK >> log2w;
  const int tiles_x = (L.nx + w - 1) >> log2w;   // block-uniform
  const int ty = t / tiles_x, tx = t - ty * tiles_x;
  x = (tx << log2w) + (int)(threadIdx.x & (w - 1));
  y = ty * h + (int)(threadIdx.x >> log2w);
  return x < L.nx && y < L.ny;
}

template <typename real>
__global__ void __launch_bounds__(BATCH_BLOCK, 6) k_batch(BatchDev B, int n_steps, int cur0) {
  __shared__ __align__(16) Lattice<real> L;
  __shared__ double red[32];
  const Lattice<real>* lat = static_cast<const Lattice<real>*>(B.lat);
  unsigned int target = 0;
  int loaded = -1;
  int w0, w1;
  for (int s = 0; s < n_steps; ++s) {
    const int cur = cur0 ^ (s & 1);
    // density
    block_range(B.n_node_tiles, w0, w1);
    for (int w = w0; w < w1; ++w) {
      const int2 t = B.node_tiles[w];
      load_lattice(L, lat, t.x, loaded);
      int x, y;
      if (tile_node(L, B.tile_log2w, t.y, x, y)) phase_rho(L, cur, x, y);
    }
    if (!grid_sync(B, ++target)) return;
    // solid layers (Eq. 15), the second after the first
    for (int layer = 1; layer <= 2; ++layer) {
      const int2* items = layer == 1 ? B.s1_items : B.s2_items;
      block_range(layer == 1 ? B.n_s1_items : B.n_s2_items, w0, w1);
      for (int w = w0; w < w1; ++w) {
        const int2 t = items[w];
        load_lattice(L, lat, t.x, loaded);
        const int j = t.y + threadIdx.x;
        if (j < (layer == 1 ? L.n_s1 : L.n_s2)) phase_solid(L, layer, j);
      }
      if (!grid_sync(B, ++target)) return;
    }
    // chemical potential (Eq. 12)
    block_range(B.n_node_tiles, w0, w1);
    for (int w = w0; w < w1; ++w) {
      const int2 t = B.node_tiles[w];
      load_lattice(L, lat, t.x, loaded);
      int x, y;
      if (L.eos != EOS_NONE && tile_node(L, B.tile_log2w, t.y, x, y)) phase_mu(L, x, y);
    }
    if (!grid_sync(B, ++target)) return;
    // force + collision + streaming
    for (int w = w0; w < w1; ++w) {
      const int2 t = B.node_tiles[w];
      load_lattice(L, lat, t.x, loaded);
      int x, y;
      if (tile_node(L, B.tile_log2w, t.y, x, y)) phase_collide(L, cur, x, y);
    }
    if (!grid_sync(B, ++target)) return;
    // boundary links (Eqs. 16-18); each chunk's compensation sum, in a fixed order
    block_range(B.n_bc_items, w0, w1);
    for (int w = w0; w < w1; ++w) {
      const int2 t = B.bc_items[w];
      load_lattice(L, lat, t.x, loaded);
      const int b = t.y + threadIdx.x;
      const double sum = b < L.n_bnodes ? phase_bc(L, cur, b) : 0.0;
      const double bs = block_sum(sum, red);
      if (threadIdx.x == 0) B.bc_partials[w] = bs;
    }
    if (!grid_sync(B, ++target)) return;
    // per-instance domain sum of the step's compensation, chunks in order
    if (threadIdx.x == 0) {
      for (int k = blockIdx.x; k < B.n_inst; k += gridDim.x) {
        double total = 0.0;
        for (int w = B.inst_bc_first[k]; w < B.inst_bc_first[k + 1]; ++w) total += B.bc_partials[w];
        const Lattice<real>& Lk = lat[k];
        const unsigned long long st = *Lk.step_ctr;
        Lk.dM_ring[st % DM_RING] = total;
        *Lk.step_ctr = st + 1;
      }
    }
  }
}

int batch_block_size() { return BATCH_BLOCK; }

long long batch_node_tiles(int nx, int ny, int log2w) {
  const int w = 1 << log2w, h = BATCH_BLOCK >> log2w;
  return (long long)((nx + w - 1) / w) * ((ny + h - 1) / h);
}

int batch_grid_size(int fp64) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (fp64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<double>, BATCH_BLOCK, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<float>, BATCH_BLOCK, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sms;
}

cudaError_t launch_batch(const BatchDev& B, int fp64, int grid, int n_steps, int cur0, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(B.bar, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  BatchDev b = B;
  void* args[] = {&b, &n_steps, &cur0};
  if (fp64)
    return cudaLaunchCooperativeKernel((const void*)k_batch<double>, dim3(grid), dim3(BATCH_BLOCK), args, 0, s);
  return cudaLaunchCooperativeKernel((const void*)k_batch<float>, dim3(grid), dim3(BATCH_BLOCK), args, 0, s);
}

}  // namespace lbmgb
