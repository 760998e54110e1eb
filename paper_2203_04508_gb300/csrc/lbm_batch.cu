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

// Copy of an instance's lattice descriptor into shared memory.  A block takes the items of a work
// list in chunks of consecutive items, which mostly belong to one instance; the copy is redone
// only when the instance changes.
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

// Items are handed out in chunks from a counter per tick and group, so that blocks whose items
// are cheap (tiles inside a cylinder, say) take more of them instead of waiting at the next
// barrier.  Three counters per group rotate over the ticks: tick tau takes counter tau % 3 and
// zeroes counter (tau + 1) % 3, which no block touches in tick tau and which the grid barrier
// publishes before tick tau + 1.
constexpr int WORK_CHUNK = 4;

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

// Row vectors of node tile t for the density and chemical-potential phases: the tile's 256 nodes
// as 256 / V vectors of V = 16/sizeof(real) consecutive nodes of a row (tile widths are at least
// 16, a multiple of V); vector u starts at (x0, y).  False outside the lattice.
template <typename real>
__device__ __forceinline__ bool tile_vec(const Lattice<real>& L, int log2w, int t, int u, int& x0, int& y) {
  constexpr int V = Vec16<real>::V;
  const int w = 1 << log2w, h = BATCH_BLOCK >> log2w, wv = w / V;
  const int tiles_x = (L.nx + w - 1) >> log2w;
  const int ty = t / tiles_x, tx = t - ty * tiles_x;
  const int row = u / wv, col = u - row * wv;
  x0 = (tx << log2w) + col * V;
  y = ty * h + row;
  return x0 < L.nx && y < L.ny;
}

// The six phases of a step, in order; the compensation sums of a step follow its boundary
// phase after a barrier.
enum { PH_RHO = 0, PH_S1, PH_S2, PH_MU, PH_COLLIDE, PH_BC, N_PHASES };
// Group 1 runs this many phases behind group 0, so that the memory-bound density pass of one
// group shares a barrier interval with the instruction-bound chemical potential of the other
// (and the collide with the first solid layer, the boundary phase with the second).
constexpr int SKEW = 3;

// work list of phase p for group g: [first, last) of the node-tile, solid-layer or
// boundary-chunk list
__device__ __forceinline__ void phase_list(const BatchDev& B, int p, int g, const int2*& items, int& first,
                                           int& last) {
  if (p == PH_S1) { items = B.s1_items; first = B.s1_start[g]; last = B.s1_start[g + 1]; }
  else if (p == PH_S2) { items = B.s2_items; first = B.s2_start[g]; last = B.s2_start[g + 1]; }
  else if (p == PH_BC) { items = B.bc_items; first = B.bc_start[g]; last = B.bc_start[g + 1]; }
  else { items = B.node_tiles; first = B.tile_start[g]; last = B.tile_start[g + 1]; }
}

// This block's share [w0, w1) of the list of phase p, for one group (block-uniform).
template <typename real>
__device__ __forceinline__ void run_phase(const BatchDev& B, const Lattice<real>* lat, Lattice<real>& L,
                                          int& loaded, int p, int cur, const int2* items, int w0, int w1,
                                          double* red) {
  int x, y;
  switch (p) {
    case PH_RHO:
    case PH_MU: {
      // row vectors (the single-lattice passes' bodies, with psi' handed from the density to the
      // chemical potential): a block takes V tiles at a time, each thread one vector of one of
      // them, whose instance's descriptor it reads from the instance table
      constexpr int V = Vec16<real>::V, U = BATCH_BLOCK / V;
      const int sub = (int)threadIdx.x / U, u = (int)threadIdx.x - sub * U;
      for (int wb = w0; wb < w1; wb += V) {
        const int w = wb + sub;
        if (w >= w1) continue;
        const int2 t = items[w];
        const Lattice<real>& Lk = lat[t.x];
        if (!tile_vec(Lk, B.tile_log2w, t.y, u, x, y)) continue;
        if (p == PH_RHO) {
          if (Lk.aa && cur == 1) {
            // one lattice in the shifted AA order: node by node through pop_index
            for (int k = 0; k < V && x + k < Lk.nx; ++k) phase_rho_pull(Lk, cur, x + k, y);
          } else {
            phase_rho_vec(Lk, cur, x, y);
          }
        } else if (Lk.eos != EOS_NONE) {
          phase_mu_vec(Lk, x, y);
        }
      }
      break;
    }
    case PH_S1:
    case PH_S2: {
      const int layer = p == PH_S1 ? 1 : 2;
      for (int w = w0; w < w1; ++w) {
        const int2 t = items[w];
        load_lattice(L, lat, t.x, loaded);
        if (layer == 2 && (t.y & BATCH_BMOM_ITEM)) {
          // one lattice in AA order: the pre-collision moments of 256 boundary nodes
          const int b = (t.y & ~BATCH_BMOM_ITEM) + (int)threadIdx.x;
          if (b < L.n_bnodes) phase_bmom(L, cur, b);
          continue;
        }
        const int j = t.y + threadIdx.x;
        if (j < (layer == 1 ? L.n_s1 : L.n_s2)) phase_solid(L, layer, j);
      }
      break;
    }
    case PH_COLLIDE:
      // per node, the stencils through L1: staging each tile's halo in shared memory (the
      // single-lattice collide kernel's way) took 27.7 against 21.6 ms per 10 steps on the
      // 256-lattice mix -- two block barriers a tile in a persistent loop without other work to
      // hide them
      // (reading each instance's descriptor from the table instead of a shared-memory copy:
      // 410 against 402 ms for 200 steps of the mix, although a block's chunks rarely share an
      // instance)
      for (int w = w0; w < w1; ++w) {
        const int2 t = items[w];
        load_lattice(L, lat, t.x, loaded);
        if (tile_node(L, B.tile_log2w, t.y, x, y)) {
          if (L.aa) phase_collide_aa(L, cur, x, y);
          else phase_collide(L, cur, x, y);
        }
      }
      break;
    default:
      // boundary links (Eqs. 16-18); each chunk's compensation sum, in a fixed order
      for (int w = w0; w < w1; ++w) {
        const int2 t = items[w];
        load_lattice(L, lat, t.x, loaded);
        const int b = t.y + threadIdx.x;
        const double sum = b < L.n_bnodes ? phase_bc(L, cur, b) : 0.0;
        const double bs = block_sum(sum, red);
        if (threadIdx.x == 0) B.bc_partials[w] = bs;
      }
  }
}

// n_steps steps of every instance.  The launch runs in ticks separated by grid barriers; at
// tick tau group g is at phase q = tau - SKEW g of its sequence (q / 6 = step, q % 6 = phase),
// so with two groups their phases interleave; with one group this is the plain lockstep
// schedule.  Each instance still runs its phases in order, so the values do not depend on the
// schedule.
template <typename real>
__global__ void __launch_bounds__(BATCH_BLOCK, 6) k_batch(BatchDev B, int n_steps, int cur0) {
  __shared__ __align__(16) Lattice<real> Ls[2];
  __shared__ double red[32];
  __shared__ int loaded[2];     // instance whose descriptor Ls[g] holds (block-uniform)
  __shared__ unsigned long long grab;   // the chunk thread 0 took
  const Lattice<real>* lat = static_cast<const Lattice<real>*>(B.lat);
  const int G = B.groups;
  const int last_q = N_PHASES * n_steps;               // q of the final compensation sums
  const int ticks = last_q + SKEW * (G - 1) + 1;
  unsigned int target = 0;
  if (threadIdx.x < 2) loaded[threadIdx.x] = -1;
  __syncthreads();
  for (int tau = 0; tau < ticks; ++tau) {
    if (tau > 0 && !grid_sync(B, ++target)) return;
    // per-instance domain sum of the compensation of the step whose boundary phase ended at
    // the barrier just passed, chunks in order
    if (threadIdx.x == 0) {
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        if (g >= G) continue;
        const int q = tau - SKEW * g;
        if (q < N_PHASES || q > last_q || q % N_PHASES != 0) continue;
        for (int k = blockIdx.x; k < B.n_inst; k += gridDim.x) {
          if (B.inst_group[k] != g) continue;
          double total = 0.0;
          for (int w = B.inst_bc[k].x; w < B.inst_bc[k].y; ++w) total += B.bc_partials[w];
          const Lattice<real>& Lk = lat[k];
          const unsigned long long st = *Lk.step_ctr;
          Lk.dM_ring[st % DM_RING] = total;
          Lk.dM_ring[DM_RING] = total;
          *Lk.step_ctr = st + 1;
        }
      }
    }
    // this tick's phase of each group; even blocks take group 0's share first, odd blocks
    // group 1's, so that every SM works on both phases at once
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int g = h ^ (int)(blockIdx.x & 1);
      const int q = tau - SKEW * g;
      if (g >= G || q < 0 || q >= last_q) continue;
      const int p = q % N_PHASES;
      const int cur = cur0 ^ ((q / N_PHASES) & 1);
      const int2* items;
      int first, last;
      phase_list(B, p, g, items, first, last);
      unsigned long long* ctr = B.work + 2 * (tau % 3) + g;
      for (;;) {
        if (threadIdx.x == 0) grab = atomicAdd(ctr, (unsigned long long)WORK_CHUNK);
        __syncthreads();
        const long long w = (long long)grab;
        __syncthreads();   // every thread has read `grab` before thread 0 takes the next chunk
        if (w >= last - first) break;   // block-uniform
        const int w1 = (int)(w + WORK_CHUNK < last - first ? w + WORK_CHUNK : last - first);
        run_phase(B, lat, Ls[g], loaded[g], p, cur, items, first + (int)w, first + w1, red);
      }
    }
    if (blockIdx.x == 0 && threadIdx.x < 2) B.work[2 * ((tau + 1) % 3) + threadIdx.x] = 0ull;
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
  if (e == cudaSuccess) e = cudaMemsetAsync(B.work, 0, BATCH_WORK_COUNTERS * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  BatchDev b = B;
  void* args[] = {&b, &n_steps, &cur0};
  if (fp64)
    return cudaLaunchCooperativeKernel((const void*)k_batch<double>, dim3(grid), dim3(BATCH_BLOCK), args, 0, s);
  return cudaLaunchCooperativeKernel((const void*)k_batch<float>, dim3(grid), dim3(BATCH_BLOCK), args, 0, s);
}

}  // namespace lbmgb
