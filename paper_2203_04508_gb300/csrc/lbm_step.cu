// Kernels of one time step and of the state set-up / read-out (sm_103a).
//
// The phases of one step, in the order of their dependencies:
//   k_rho_vec       density of every fluid node from the 9 offset populations   (Sec. 2.1),
//                   and the pointwise part of Eq. 12, psi'(rho) (or psi, pseudopotential force)
//   k_solid (x2)    densities of the first, then second solid layer             (Eq. 15)
//   k_mu_sweep      chemical potential at fluid nodes by row sweeps (large FP32  (Eq. 12)
//                   lattices; k_mu_vec by row vectors otherwise, k_mu per node where psi' is
//                   not supplied; k_psi for the pseudopotential force outside the overlapped
//                   step)
//   k_collide_tma / k_collide
//                   force (Eq. 9) + collision (Eq. 4) + exact-difference forcing (Eq. 13)
//                   + push streaming (Eq. 5) into the other lattice: TMA-pipelined persistent
//                   kernel on large FP32 lattices, one tile per block otherwise
//   k_bc            every cut link by Eq. 16 / Eq. 17, the per-node compensation of Eq. 18
//                   accumulated in FP64, and the deterministic domain sum of that step
// launch_step issues them one after another on one stream (used by the reverse sweep's
// recomputation and by the per-phase timing).  lbm_step uses launch_step_overlap instead: the
// step starts at the chemical potential (none for the pseudopotential force, whose psi the
// previous step formed), and after the collide the next state's density pass runs on a second
// stream while k_bc and the next state's solid layers run on the first (same values).
// The per-node bodies of the phases live in lbm_phases.cuh.
#include <algorithm>
#include <cstdio>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_phases.cuh"

namespace lbmgb {

constexpr int NODE_BLOCK = 256;

// node kernels run on a 2D grid of TILE_X x TILE_Y blocks: x along the row, y across rows
constexpr int TILE_X = 128, TILE_Y = 2;

template <typename real>
__device__ __forceinline__ bool node_of_thread(const Lattice<real>& L, int& x, int& y, int& n) {
  x = blockIdx.x * TILE_X + threadIdx.x;
  y = blockIdx.y * TILE_Y + threadIdx.y;
  n = y * L.pitch + x;
  return x < L.nx && y < L.ny;
}

// Density pass with 16-byte loads: each thread takes V = 16/sizeof(real) consecutive nodes of
// a row (phase_rho_vec).  Rows are taken from the top down: the collide kernel writes the new
// populations roughly from the bottom up, so the rows it wrote last are still in L2 when this pass
// starts, and the rows this pass reads last are the ones the next collide reads first.
// FP32: five blocks an SM (48 registers, 8 bytes spilled) instead of four (56): 0.0590 -> 0.0583 ms
// on the 2048 x 4096 impact lattice.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK, sizeof(real) == 4 ? 5 : 1) k_rho_vec(Lattice<real> L, int cur) {
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * Vec16<real>::V, y = L.ny - 1 - (int)blockIdx.y;
  if (x0 < L.nx) phase_rho_vec(L, cur, x0, y);
}

// The density pass of a state in AA order (one lattice after its in-place step): f_i(x) lies in
// slot opp(i) of x - e_i, so the rows are shifted per direction and the 16-byte loads of
// k_rho_vec do not apply; one node a thread, the same sums and stores as k_rho_vec.  (A row-vector
// variant -- aligned vectors plus one element from the neighbouring lane by a shuffle -- took
// 75.9 against 66.8 us on the 2048 x 4096 lattice: 64 registers, and the warp-edge lanes' extra
// dependent loads.)
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_rho_pull(Lattice<real> L, int cur) {
  // rows from the top down, as k_rho_vec takes them
  const int x = blockIdx.x * TILE_X + threadIdx.x, y = L.ny - 1 - (int)(blockIdx.y * TILE_Y + threadIdx.y);
  if (x < L.nx && y >= 0) phase_rho_pull(L, cur, x, y);
}

// One lattice (AA order): the pre-collision moments of every boundary node, which the boundary
// phase needs after the collide has overwritten the populations (the sums of `moments`).
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_bmom(Lattice<real> L, int cur) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < L.n_bnodes) phase_bmom(L, cur, b);
}

// psi(rho_s) (1 + c_w) of a solid-layer node whose density is rho_s (pseudopotential force)
template <typename real>
__device__ __forceinline__ real psi_wall(const Lattice<real>& L, int n, real rs) {
  const int b = L.body[n];
  const double cw = b < L.n_cyl ? L.cyl[4 * b + 3] : L.cw_walls;
  return psi_of(L, rs) * (real(1) + (real)cw);
}

// Eq. 15 for one solid layer; with the pseudopotential force also the layer's psi, so that the
// psi plane of the state is complete without a separate pass
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_solid(Lattice<real> L, int layer) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (layer == 1 ? L.n_s1 : L.n_s2)) return;
  phase_solid(L, layer, j);
  if (L.pseudo && L.eos != EOS_NONE) {
    const int n = layer == 1 ? L.s1node[j] : L.s2node[j];
    L.mu[n] = psi_wall(L, n, L.rho[n]);
  }
}


template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_mu(Lattice<real> L) {
  int x, y, n;
  if (!node_of_thread(L, x, y, n)) return;
  if (L.psip) {
    // phase_mu with psi'(rho) - mu_sat from the density pass: the same value, the same sum
    if (L.kind[n] != KIND_FLUID) return;
    Stencil st = stencil_at(L, x, y);
    L.mu[n] = mu_of(L, L.psip[n], lap4(L.rho, n, st));
    return;
  }
  phase_mu(L, x, y);
}

// The chemical-potential pass with psi' from the density pass, V = 16/sizeof(real) consecutive
// nodes of a row per thread (phase_mu_vec).
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_mu_vec(Lattice<real> L) {
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * Vec16<real>::V, y = blockIdx.y;
  if (x0 < L.nx) phase_mu_vec(L, x0, y);
}

// cp.async (an asynchronous 16- or 4-byte copy into shared memory, completed by groups); a
// source size of 0 writes zeros and reads nothing
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Chemical potential (FP32) by row sweeps: a thread holds four consecutive nodes of a row and
// walks MU_ROWS rows down its column, keeping the five rows of the 9-point stencil in registers,
// so that a row costs it one density vector, one psi' vector and the node classes.  Those three
// arrive by cp.async into the thread's own shared-memory slots, MU_DEPTH rows ahead (the loads
// in flight hold no registers).  The centre row's two further nodes on each side come from the
// neighbouring lanes; lanes at a warp's edge, at the lattice's x edges or at a ragged end load
// them one by one with the periodic wrap.  Same values and the same sums as k_mu (lap4_of,
// mu_of).
// Rows a thread walks, threads a block (a 512-node strip) and rows in flight.  On the
// 2048 x 4096 impact lattice: 4 x 128 x 4 0.0243 ms, 8 x 128 x 4 (or 6) 0.0246, 16 x 128 x 4
// 0.0250, 8 and 16 rows with 8 in flight 0.027 and 0.031; with the loads in registers one row
// ahead the best was 0.0265 and with the classes and psi' not ahead 0.030.
constexpr int MU_ROWS = 4, MU_BLOCK = 128, MU_DEPTH = 4;
__global__ void __launch_bounds__(MU_BLOCK) k_mu_sweep(Lattice<float> L) {
  __shared__ float4 s_rho[MU_DEPTH][MU_BLOCK];
  __shared__ float4 s_psi[MU_DEPTH][MU_BLOCK];
  __shared__ uchar4 s_kind[MU_DEPTH][MU_BLOCK];
  const int t = threadIdx.x, lane = t & 31;
  const int x0 = (blockIdx.x * blockDim.x + t) * 4;
  const int ya = blockIdx.y * MU_ROWS, yb = min(ya + MU_ROWS, L.ny);
  const bool live = x0 < L.nx, full = x0 + 4 <= L.nx;
  const float* __restrict__ r = L.rho;
  // this thread's vector of row y (zeros beyond a wall, wrapped on a periodic lattice)
  auto row = [&](int y) -> float4 {
    if (!live) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (y < 0 || y >= L.ny) {
      if (L.walls) return make_float4(0.f, 0.f, 0.f, 0.f);
      y = y < 0 ? y + L.ny : y - L.ny;
    }
    return __ldg(reinterpret_cast<const float4*>(r + y * L.pitch + x0));
  };
  // group j: the classes and psi' of row ya + j and the density of row ya + j + 3 (which the
  // last row of the sweep does not need), into slot j % MU_DEPTH
  auto issue = [&](int j) {
    const int y = ya + j;
    if (y < yb) {
      const int slot = j % MU_DEPTH;
      const long long n0 = (long long)y * L.pitch + (live ? x0 : 0);
      cp_async4(&s_kind[slot][t], L.kind + n0, live ? 4 : 0);
      cp_async16(&s_psi[slot][t], L.psip + n0, live ? 16 : 0);
      int yr = y + 3;
      bool ok = live && y + 1 < yb;
      if (yr >= L.ny) {
        if (L.walls) ok = false;
        else yr -= L.ny;
      }
      cp_async16(&s_rho[slot][t], r + (ok ? (long long)yr * L.pitch + x0 : 0), ok ? 16 : 0);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int j = 0; j < MU_DEPTH; ++j) issue(j);
  float4 w0 = row(ya - 2), w1 = row(ya - 1), w2 = row(ya), w3 = row(ya + 1), w4 = row(ya + 2);
  // lanes whose centre-row neighbours the next lanes hold
  const bool left_ok = lane > 0 && full;
  const bool right_ok = lane < 31 && x0 + 6 <= L.nx;
  for (int y = ya; y < yb; ++y) {
    const int j = y - ya, slot = j % MU_DEPTH;
    cp_async_wait<MU_DEPTH - 1>();
    const uchar4 kind = s_kind[slot][t];
    const float4 pp = s_psi[slot][t];
    const float4 ahead = s_rho[slot][t];
    issue(j + MU_DEPTH);
    const int n0 = y * L.pitch + x0;
    const float lz = __shfl_up_sync(0xffffffffu, w2.z, 1), lw = __shfl_up_sync(0xffffffffu, w2.w, 1);
    const float rx = __shfl_down_sync(0xffffffffu, w2.x, 1), ry = __shfl_down_sync(0xffffffffu, w2.y, 1);
    const bool fl[4] = {kind.x == KIND_FLUID && x0 < L.nx, kind.y == KIND_FLUID && x0 + 1 < L.nx,
                        kind.z == KIND_FLUID && x0 + 2 < L.nx, kind.w == KIND_FLUID && x0 + 3 < L.nx};
    if (fl[0] || fl[1] || fl[2] || fl[3]) {
      float c[8];   // the centre row, x0 - 2 .. x0 + 5
      const int rb = y * L.pitch;
      if (full) {
        c[2] = w2.x; c[3] = w2.y; c[4] = w2.z; c[5] = w2.w;
      } else {
#pragma unroll
        for (int j2 = 2; j2 < 6; ++j2) c[j2] = r[rb + wrap_x(L, x0 - 2 + j2)];
      }
      if (left_ok) { c[0] = lz; c[1] = lw; }
      else { c[0] = r[rb + wrap_x(L, x0 - 2)]; c[1] = r[rb + wrap_x(L, x0 - 1)]; }
      if (right_ok && full) { c[6] = rx; c[7] = ry; }
      else { c[6] = r[rb + wrap_x(L, x0 + 4)]; c[7] = r[rb + wrap_x(L, x0 + 5)]; }
      const float up1[4] = {w3.x, w3.y, w3.z, w3.w}, dn1[4] = {w1.x, w1.y, w1.z, w1.w};
      const float up2[4] = {w4.x, w4.y, w4.z, w4.w}, dn2[4] = {w0.x, w0.y, w0.z, w0.w};
      const float ps[4] = {pp.x, pp.y, pp.z, pp.w};
      float m[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = k + 2;
        m[k] = mu_of(L, ps[k], lap4_of(c[i], c[i + 1], c[i - 1], c[i + 2], c[i - 2], up1[k], dn1[k], up2[k], dn2[k]));
      }
      if (fl[0] && fl[1] && fl[2] && fl[3]) {
        *reinterpret_cast<float4*>(L.mu + n0) = make_float4(m[0], m[1], m[2], m[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (fl[k]) L.mu[n0 + k] = m[k];
      }
    }
    w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = ahead;
  }
  cp_async_wait<0>();
}

// The next state's density and chemical potential in one pass (FP32, chemical-potential force;
// lbm_set_mu_kernel 3).  A block takes a tile of RM_W x RM_H nodes: it forms the density of the
// tile and a halo of RM_HX columns and RM_HY rows from the populations into shared memory
// (16-byte loads; wrapped or scalar at the lattice's edges), stores the tile's fluid densities,
// and then each thread walks one column of the tile, evaluating Eq. 12 from the staged
// densities -- psi'(rho) - mu_sat by psi_prime_shifted, the Laplacian by lap4_of, mu by mu_of,
// the operations of the density and chemical-potential passes, so the values are theirs.  The
// halo densities are those of the populations as they are now; where a node's stencil reaches
// a boundary node (whose populations the boundary phase is still changing) or a solid node
// (whose density the solid-layer kernels form), its mu is recomputed from the final density
// plane by k_mu_near after the boundary phase.  Saves the chemical-potential pass at the start
// of the next step.
constexpr int RM_W = 256, RM_H = 32, RM_HX = 4, RM_HY = 2;
constexpr int RM_SW = RM_W + 2 * RM_HX, RM_SH = RM_H + 2 * RM_HY;
static_assert(RM_HX % 4 == 0 && RM_HX >= 2 && RM_HY >= 2, "the halo covers the stencil in whole vectors");
__global__ void __launch_bounds__(NODE_BLOCK) k_rho_mu_tile(Lattice<float> L, int cur) {
  __shared__ __align__(16) float s_rho[RM_SH][RM_SW];
  __shared__ __align__(16) uint8_t s_kind[RM_H][RM_W];   // the tile's node classes, for the second phase
  const int x0 = blockIdx.x * RM_W, y0 = blockIdx.y * RM_H;
  const float* __restrict__ f = L.f[cur];
  constexpr int GX = RM_SW / 4;
  for (int g = threadIdx.x; g < GX * RM_SH; g += NODE_BLOCK) {
    const int gy = g / GX, gx = g - gy * GX;
    const int y = y0 - RM_HY + gy, xs = x0 - RM_HX + 4 * gx;
    // rows beyond a wall read as zero; a periodic lattice wraps (however small it is)
    int yy = y;
    bool row_ok = true;
    if (yy < 0 || yy >= L.ny) {
      if (L.walls) row_ok = false;
      else yy = ((yy % L.ny) + L.ny) % L.ny;
    }
    float r[4] = {0.f, 0.f, 0.f, 0.f};
    if (row_ok) {
      const int rb = yy * L.pitch;
      if (xs >= 0 && xs + 4 <= L.nx) {
        float4 fv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) fv[i] = __ldg(reinterpret_cast<const float4*>(f + i * L.plane + rb + xs));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float fl[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) fl[i] = lane_of<float>(fv[i], k);
          r[k] = density_of(L, fl);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int x = ((xs + k) % L.nx + L.nx) % L.nx;   // x is periodic
          float fl[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) fl[i] = f[i * L.plane + rb + x];
          r[k] = density_of(L, fl);
        }
      }
    }
    *reinterpret_cast<float4*>(&s_rho[gy][4 * gx]) = make_float4(r[0], r[1], r[2], r[3]);
    // the tile's own fluid densities (a solid node's slot belongs to the solid-layer kernels,
    // which may be writing it now: vectors with one take the scalar path)
    if (gy >= RM_HY && gy < RM_HY + RM_H && gx >= RM_HX / 4 && gx < (RM_HX + RM_W) / 4) {
      uchar4 kd = make_uchar4(KIND_PAD, KIND_PAD, KIND_PAD, KIND_PAD);
      if (y < L.ny && xs < L.nx) kd = __ldg(reinterpret_cast<const uchar4*>(L.kind + y * L.pitch + xs));
      *reinterpret_cast<uchar4*>(&s_kind[gy - RM_HY][xs - x0]) = kd;
    }
    if (gy >= RM_HY && gy < RM_HY + RM_H && gx >= RM_HX / 4 && gx < (RM_HX + RM_W) / 4 && y < L.ny && xs < L.nx) {
      const int n0 = y * L.pitch + xs;
      const uchar4 kd = *reinterpret_cast<const uchar4*>(&s_kind[gy - RM_HY][xs - x0]);
      const bool fl[4] = {kd.x == KIND_FLUID, kd.y == KIND_FLUID && xs + 1 < L.nx, kd.z == KIND_FLUID && xs + 2 < L.nx,
                          kd.w == KIND_FLUID && xs + 3 < L.nx};
      if (fl[0] && fl[1] && fl[2] && fl[3]) {
        *reinterpret_cast<float4*>(L.rho + n0) = make_float4(r[0], r[1], r[2], r[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (fl[k]) L.rho[n0 + k] = r[k];
      }
    }
  }
  __syncthreads();
  const int x = x0 + threadIdx.x;
  if (x >= L.nx) return;
  const int cx = RM_HX + threadIdx.x;
  float dn2 = s_rho[0][cx], dn1 = s_rho[1][cx], c = s_rho[2][cx], up1 = s_rho[3][cx];
  for (int j = 0; j < RM_H; ++j) {
    const int y = y0 + j;
    if (y >= L.ny) break;
    const float up2 = s_rho[j + 4][cx];
    const int n = y * L.pitch + x;
    if (s_kind[j][threadIdx.x] == KIND_FLUID) {
      const float* row = s_rho[j + RM_HY];
      const float lap = lap4_of(c, row[cx + 1], row[cx - 1], row[cx + 2], row[cx - 2], up1, dn1, up2, dn2);
      L.mu[n] = mu_of(L, psi_prime_shifted(L, c), lap);
    }
    dn2 = dn1; dn1 = c; c = up1; up1 = up2;
  }
}

// Chemical potential of the listed fluid nodes from the final density plane (k_mu's
// arithmetic, psi' evaluated here): the nodes k_rho_mu_tile could not finish.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_mu_near(Lattice<real> L) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.n_near) return;
  const int n = L.near_list[j];
  const int x = n % L.pitch, y = n / L.pitch;
  Stencil st = stencil_at(L, x, y);
  L.mu[n] = mu_of(L, psi_prime_shifted(L, L.rho[n]), lap4(L.rho, n, st));
}

// Pseudopotential force model: psi(rho) at fluid nodes, psi(rho_s) (1 + c_w) at the two solid
// layers (rho_s from Eq. 15, c_w the wall factor of the node's body).  Pointwise, so it takes
// V consecutive nodes of a row per thread with one 16-byte density load, like k_rho_vec.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_psi(Lattice<real> L) {
  using VT = typename Vec16<real>::type;
  constexpr int V = Vec16<real>::V;
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * V, y = blockIdx.y;
  if (x0 >= L.nx) return;
  const int n0 = y * L.pitch + x0;
  const VT rv = __ldg(reinterpret_cast<const VT*>(L.rho + n0));
#pragma unroll
  for (int k = 0; k < V; ++k) {
    if (x0 + k >= L.nx) break;
    const uint8_t kd = L.kind[n0 + k];
    if (kd == KIND_FLUID || kd == KIND_SOLID1 || kd == KIND_SOLID2) {
      real v = psi_of(L, lane_of<real>(rv, k));
      if (kd != KIND_FLUID) {
        const int b = L.body[n0 + k];
        const double cw = b < L.n_cyl ? L.cyl[4 * b + 3] : L.cw_walls;
        v *= real(1) + (real)cw;
      }
      L.mu[n0 + k] = v;
    }
  }
}

static_assert(CT_X * CT_Y == NODE_BLOCK, "a collide tile is one node a thread");

// Force + collision + streaming.  A block of 32 x 8 nodes (one warp per 128-byte row) first
// stages the density and chemical potential of its tile and of a two-node halo in shared
// memory (stage_tile), so that the fourth-order gradients of Eq. 9 read 16 neighbours there
// instead of through the L1/L2 path; the arithmetic is force_at's, operation for operation.
// PSEUDO: the pseudopotential force from the staged psi tile (its one-node halo); no density
// staging.

// LAY: 0 two lattices; one lattice in AA order, 1 its first step (natural order in, each node's
// own slots rewritten in place), 2 its second (f_i(x) pulled from slot opp(i) of x - e_i, pushed
// into slot i of x + e_i).
template <typename real, bool PSEUDO, int LAY = 0>
__global__ void __launch_bounds__(NODE_BLOCK) k_collide(Lattice<real> L, int cur) {
  __shared__ real s_rho[CT_SY][CT_SX];
  __shared__ real s_mu[CT_SY][CT_SX];
  const int x0 = blockIdx.x * CT_X, y0 = blockIdx.y * CT_Y;
  const bool stencils = L.eos != EOS_NONE;
  const int lx = threadIdx.x % CT_X, ly = threadIdx.x / CT_X;
  const int x = x0 + lx, y = y0 + ly;
  // the node's own populations are requested before the halo, so both loads are in flight
  // together
  const bool fluid = x < L.nx && y < L.ny && L.kind[y * L.pitch + x] == KIND_FLUID;
  real fl[9];
  if (fluid) {
    if (LAY == 2) {
      const real* fin = L.f[0];
      const int n = y * L.pitch + x;
      if (interior(L, x, y)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) fl[i] = fin[opp(i) * L.plane + n - ex(i) - ey(i) * L.pitch];
      } else {
        load_pops(L, 1, x, y, fl);
      }
    } else {
      const real* __restrict__ fin = L.f[cur];
#pragma unroll
      for (int i = 0; i < 9; ++i) fl[i] = fin[i * L.plane + y * L.pitch + x];
    }
  }
  if (stencils) {
    stage_tile<real, PSEUDO>(L, x0, y0, s_rho, s_mu);
    __syncthreads();
  }
  if (!fluid) return;
  real g[4] = {real(0), real(0), real(0), real(0)};
  if (stencils) tile_force_terms<real, PSEUDO>(&s_mu[0][0], &s_rho[0][0], CT_SX, (ly + CT_H) * CT_SX + lx + CT_H, g);
  collide_loaded<LAY == 1>(L, cur, x, y, fl,
                           [&](real r, real& Fx, real& Fy) { tile_force<real, PSEUDO>(L, stencils, g, r, Fx, Fy); });
}

// ---------------------------------------------------------------------------------------
// Force + collision + streaming, TMA-pipelined (FP32).  A persistent grid; each block walks the
// 32 x 8 tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...  Per tile, cp.async.bulk.tensor loads
// complete on the stage's mbarrier: one 3D load brings the nine population planes (9 KB), 2D
// loads the density and chemical-potential tile with its two-node halo (chemical-potential
// force), or the psi tile (pseudopotential force, whose stencil reaches one node), as 40 x 12
// boxes from x0 - 4 so that the first coordinate stays on a 16-byte boundary.  TMA_STAGES
// stages: while the block computes tile k, the loads of the next tiles are in flight.  Tiles
// whose halo wraps around a periodic edge stage it with plain loads instead (the TMA fill
// value is zero, not the wrapped node).  Per node the arithmetic is k_collide's (the same
// force terms, assembled in the same rounding order), so both kernels give the same bits.
// Every mbarrier wait is bounded: a block that gives up sets L.kerr, waits (bounded) for its
// own copies and returns.
// ---------------------------------------------------------------------------------------
constexpr int TMA_STAGES = 2;
constexpr int TMA_HX = 40, TMA_HOX = 4;            // width and x offset of the halo boxes
constexpr int TMA_MY = CT_Y + 2 * CT_H;            // their rows (a two-node halo)
constexpr int TMA_F_BYTES = 9 * CT_Y * CT_X * 4;
constexpr int TMA_M_BYTES = TMA_HX * TMA_MY * 4;
// stage: populations, then density and mu (chemical potential) or psi (pseudopotential)
constexpr int TMA_STAGE_CP = TMA_F_BYTES + 2 * TMA_M_BYTES;
constexpr int TMA_STAGE_PP = TMA_F_BYTES + TMA_M_BYTES;
constexpr long long TMA_SPIN_LIMIT = 1 << 22;
static_assert(TMA_F_BYTES % 128 == 0 && TMA_M_BYTES % 128 == 0, "stage buffers stay 128-byte aligned");
static_assert((TMA_HOX * 4) % 16 == 0 && (CT_X * 4) % 16 == 0 && (TMA_HX * 4) % 16 == 0,
              "TMA boxes start and extend on 16-byte boundaries");
static_assert(TMA_HOX >= CT_H && TMA_HX - TMA_HOX >= CT_X + CT_H, "the boxes cover the halo the stencils read");
// The second step of the AA order pulls f_i(x) from slot opp(i) of x - e_i: a 40 x 10 x 9 box from
// (x0 - 4, y0 - 1) covers every shifted row of a tile (its x start stays on a 16-byte boundary).
constexpr int TMA_PX = 40, TMA_POX = 4, TMA_PY = CT_Y + 2;
constexpr int TMA_FP_BOX = 9 * TMA_PY * TMA_PX * 4;                 // bytes the box delivers
constexpr int TMA_FP_BYTES = (TMA_FP_BOX + 127) / 128 * 128;        // its stage area
static_assert((TMA_POX * 4) % 16 == 0 && (TMA_PX * 4) % 16 == 0 && TMA_PX - TMA_POX >= CT_X + 1 && TMA_POX >= 1,
              "the pull box covers a tile shifted by one node and starts on a 16-byte boundary");

// FMODE: 0 push into the other lattice, 1 in place (the AA order's first step), 2 pulled from
// the shifted slots and pushed (its second step)
__host__ __device__ constexpr int tma_stage_bytes(bool pseudo, int fmode = 0) {
  return (fmode == 2 ? TMA_FP_BYTES : TMA_F_BYTES) + (pseudo ? 1 : 2) * TMA_M_BYTES;
}

struct CollideMaps {
  CUtensorMap f;      // populations of the input lattice, box 32 x 8 x 9
  CUtensorMap rho;    // density plane, box 40 x 12
  CUtensorMap mu;     // chemical-potential (psi) plane, box 40 x 12
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity to complete (at most `limit` polls)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = TMA_SPIN_LIMIT) {
  for (long long it = 0; it < limit; ++it) {
    if (mbar_test(bar, parity)) return true;
    if (it > 8) __nanosleep(32);
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// does every halo node the tile's stencils read lie inside the lattice (no periodic wrap), so
// that TMA can fetch it?  Two nodes out for Eq. 9, one for the pseudopotential force.
template <bool PSEUDO>
__device__ __forceinline__ bool tma_halo(const Lattice<float>& L, int x0, int y0) {
  const int h = PSEUDO ? 1 : CT_H;
  return x0 - h >= 0 && x0 + CT_X + h <= L.nx && (L.walls || (y0 - h >= 0 && y0 + CT_Y + h <= L.ny));
}

// Column sweeps (SWEEP): the same force + collision + streaming, and the next state's density
// with it (FP32, chemical-potential force, lattices of whole 32 x 8 tiles).  Block (strip,
// band) walks the tiles of one 32-column strip upwards through a band of tile rows, and drops
// each post-collision population, besides pushing it into the other lattice, into a
// shared-memory ring at its destination: ring rows are destination rows (row - ya + 1) mod
// SW_R of the band [ya, yb), ring columns x0 - 1 .. x0 + 32.  Once tile y0 has collided, rows
// y0 - 1 .. y0 + 6 hold every population streaming into them, and the block sums them in the
// density pass's order (density_sum) into the density and psi'(rho) - mu_sat of the strip's
// inner 30 columns.  k_rho_sweep_fix finishes the rest: the strip's two edge columns, whose
// incoming populations come partly from the neighbouring strips -- every block leaves the
// values it holds for its own edge nodes and for its neighbours' in the edge buffer -- and the
// band's first and last rows, whose neighbours across the band edge another block collides.
// Boundary nodes' values are provisional, as in the density pass: the boundary phase changes
// their populations and k_rho_scatter stores their final density.
constexpr int SW_R = CT_Y + 2;                       // ring rows
constexpr int SW_W = CT_X + 2;                       // ring columns
constexpr int SW_RING_BYTES = 9 * SW_R * SW_W * 4;
constexpr int SW_KIND_BYTES = SW_R * CT_X;
static_assert(18 * CT_Y <= NODE_BLOCK, "one thread per edge-buffer entry of a tile");

__host__ __device__ constexpr size_t collide_smem_bytes(bool pseudo, bool sweep, int fmode = 0) {
  return (size_t)TMA_STAGES * tma_stage_bytes(pseudo, fmode) + (sweep ? (size_t)SW_RING_BYTES + SW_KIND_BYTES : 0);
}

// first tile row of band b of `bands` over `tile_rows` tile rows
__host__ __device__ inline int sweep_band_start(int b, int bands, int tile_rows) {
  return (int)((long long)b * tile_rows / bands);
}

struct SweepArgs {
  float* rho_next;   // the next state's density plane
  float* edge;       // edge buffer: direction i, edge column c, row y at (i * 2 strips + c) * ny + y;
                     // edge column 2 s is strip s's first column, 2 s + 1 its last
  int strips, bands, tile_rows;
};

// entry e (0..17) of one row of a strip's edge values: its direction, ring column and edge column.
// 0-5: the strip's first column (directions arriving from inside the strip); 6-8: the column
// left of the strip (directions leaving to the left); 9-14: the strip's last column; 15-17: the
// column right of the strip.
__device__ __forceinline__ void sweep_edge_entry(int e, int strip, int strips, int& dir, int& rcol, int& ecol) {
  dir = (int)((e < 9 ? (0x763764320ULL >> (4 * e)) : (0x851854210ULL >> (4 * (e - 9)))) & 15ULL);
  if (e < 6) { rcol = 1; ecol = 2 * strip; }
  else if (e < 9) { rcol = 0; ecol = 2 * (strip == 0 ? strips - 1 : strip - 1) + 1; }
  else if (e < 15) { rcol = CT_X; ecol = 2 * strip + 1; }
  else { rcol = CT_X + 1; ecol = 2 * (strip + 1 == strips ? 0 : strip + 1); }
}

// One lattice in AA order: FMODE 1, its first step -- tiles are loaded as in natural order and
// every node's post-collision populations go back into its own slots (collide_loaded); FMODE 2,
// its second -- M.f is the 40 x 10 x 9 pull box, each node reads f_i from slot opp(i) of x - e_i
// in it (tiles whose shifted rows wrap around an edge read them from global memory) and pushes
// into the same lattice.
template <bool PSEUDO, bool SWEEP, int FMODE = 0>
__global__ void __launch_bounds__(NODE_BLOCK) k_collide_tma(Lattice<float> L, int cur, const __grid_constant__ CollideMaps M,
                                                            int tiles_x, int n_tiles, SweepArgs A) {
  static_assert(!(PSEUDO && SWEEP), "the sweep forms the chemical-potential model's density");
  static_assert(!(SWEEP && FMODE != 0), "the sweep pushes into a second lattice");
  constexpr int FB = FMODE == 2 ? TMA_FP_BYTES : TMA_F_BYTES;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ __align__(8) uint64_t bar[TMA_STAGES];
  // per stage, set by the thread that requests its tile: x0, y0, and flags (1: the halo came by
  // TMA, 2: no push of the tile wraps around an edge)
  __shared__ int4 info[TMA_STAGES];
  constexpr int SB = tma_stage_bytes(PSEUDO, FMODE);
  const bool stencils = L.eos != EOS_NONE;
  const int lx = threadIdx.x % CT_X, ly = threadIdx.x / CT_X;
  auto f_of = [&](int s) { return reinterpret_cast<float*>(tma_smem + s * SB); };
  // mu (or psi) right after the populations, the density (chemical potential) after it
  auto mu_of = [&](int s) { return reinterpret_cast<float*>(tma_smem + s * SB + FB); };
  auto rho_of = [&](int s) { return reinterpret_cast<float*>(tma_smem + s * SB + FB + TMA_M_BYTES); };
  float* ring = reinterpret_cast<float*>(tma_smem + TMA_STAGES * SB);
  uint8_t* rkind = tma_smem + TMA_STAGES * SB + SW_RING_BYTES;
  // this block's tiles k = 0 .. nt - 1, as tile coordinates (tx, ty) advanced without a division:
  // tiles blockIdx.x + k gridDim.x of the row-major tile order, or its band of one strip
  int nt, ya = 0, tx, ty, dx = 0, dy = 1;
  if (SWEEP) {
    tx = blockIdx.x % A.strips;
    const int band = blockIdx.x / A.strips;
    const int tr0 = sweep_band_start(band, A.bands, A.tile_rows);
    nt = sweep_band_start(band + 1, A.bands, A.tile_rows) - tr0;
    ty = tr0;
    ya = tr0 * CT_Y;
  } else {
    nt = n_tiles > (int)blockIdx.x ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    tx = (int)blockIdx.x % tiles_x;
    ty = (int)blockIdx.x / tiles_x;
    dx = (int)gridDim.x % tiles_x;
    dy = (int)gridDim.x / tiles_x;
  }
  auto advance = [&](int& ax, int& ay) {
    ax += dx;
    ay += dy;
    if (ax >= tiles_x && !SWEEP) {
      ax -= tiles_x;
      ++ay;
    }
  };
  int itx = tx, ity = ty;   // thread 0: the next tile to request
  // thread 0: request the next tile into stage s
  auto issue = [&](int s) {
    const int x0 = itx * CT_X, y0 = ity * CT_Y;
    advance(itx, ity);
    const bool h = stencils && tma_halo<PSEUDO>(L, x0, y0);
    // with walls, rows never wrap
    const bool inner = x0 >= 1 && x0 + CT_X < L.nx && (L.walls || (y0 >= 1 && y0 + CT_Y < L.ny));
    info[s] = make_int4(x0, y0, (h ? 1 : 0) | (inner ? 2 : 0), 0);
    mbar_expect_tx(&bar[s], (FMODE == 2 ? TMA_FP_BOX : TMA_F_BYTES) + (h ? (PSEUDO ? 1 : 2) * TMA_M_BYTES : 0));
    if (FMODE == 2) tma_load_3d(f_of(s), &M.f, x0 - TMA_POX, y0 - 1, 0, &bar[s]);
    else tma_load_3d(f_of(s), &M.f, x0, y0, 0, &bar[s]);
    if (h) {
      tma_load_2d(mu_of(s), &M.mu, x0 - TMA_HOX, y0 - CT_H, &bar[s]);
      if (!PSEUDO) tma_load_2d(rho_of(s), &M.rho, x0 - TMA_HOX, y0 - CT_H, &bar[s]);
    }
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < TMA_STAGES; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < TMA_STAGES && s < nt; ++s) issue(s);
  }
  __syncthreads();
  for (int k = 0; k < nt; ++k) {
    const int s = k % TMA_STAGES;
    const int4 tile = info[s];
    const int x0 = tile.x, y0 = tile.y;
    const bool inner = (tile.z & 2) != 0;
    const int x = x0 + lx, y = y0 + ly;
    const bool fluid = x < L.nx && y < L.ny && L.kind[y * L.pitch + x] == KIND_FLUID;
    // a wait that gives up is acted on at the block barrier below, once every thread has read
    // the stage (what a thread whose wait gave up read is never used)
    const bool ok = mbar_wait(&bar[s], (uint32_t)((k / TMA_STAGES) & 1), L.spin_limit);
    float* sm = mu_of(s);
    float* sr = rho_of(s);
    if (stencils && !(tile.z & 1)) {
      // the halo wraps around a periodic edge: plain wrap-aware loads, as k_collide stages it
      const int h = PSEUDO ? 1 : CT_H;
      for (int e = threadIdx.x; e < TMA_HX * TMA_MY; e += NODE_BLOCK) {
        const int ey = e / TMA_HX, ex = e - ey * TMA_HX;
        const int xx = x0 + ex - TMA_HOX, yy = y0 + ey - CT_H;
        float r = 0.0f, m = 0.0f;
        if (xx >= -h && xx <= L.nx + h - 1 && (L.walls ? (yy >= 0 && yy < L.ny) : (yy >= -h && yy <= L.ny + h - 1))) {
          const int n = node_at(L, xx, yy);
          if (!PSEUDO) r = L.rho[n];
          m = L.mu[n];
        }
        if (!PSEUDO) sr[e] = r;
        sm[e] = m;
      }
      __syncthreads();
    }
    float fl[9];
    float g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (fluid) {
      const float* sf = f_of(s);
      if (FMODE == 2) {
        if (inner) {
#pragma unroll
          for (int i = 0; i < 9; ++i) fl[i] = sf[(opp(i) * TMA_PY + ly + 1 - ey(i)) * TMA_PX + lx + TMA_POX - ex(i)];
        } else {
          load_pops(L, 1, x, y, fl);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) fl[i] = sf[(i * CT_Y + ly) * CT_X + lx];
      }
      if (stencils) tile_force_terms<float, PSEUDO>(sm, sr, TMA_HX, (ly + CT_H) * TMA_HX + lx + TMA_HOX, g);
    }
    // every thread has read stage s: refill it with the tile TMA_STAGES ahead -- or give up:
    // flag it, let this block's copies still in flight land, and leave
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(L.kerr, 1u);
        for (int j = 0; j < TMA_STAGES && k + j < nt; ++j)
          mbar_wait(&bar[(k + j) % TMA_STAGES], (uint32_t)(((k + j) / TMA_STAGES) & 1));
      }
      __syncthreads();
      return;
    }
    if (threadIdx.x == 0 && k + TMA_STAGES < nt) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(s);
    }
    if (!SWEEP) {
      if (!fluid) continue;
      collide_loaded<FMODE == 1>(
          L, cur, x, y, fl, [&](float r, float& Fx, float& Fy) { tile_force<float, PSEUDO>(L, stencils, g, r, Fx, Fy); },
          inner);
      continue;
    }
    // ring rows of this node's row and of the rows below and above it
    const int sc = (y - ya + 1) % SW_R;
    const int sm1 = sc == 0 ? SW_R - 1 : sc - 1, sp1 = sc == SW_R - 1 ? 0 : sc + 1;
    rkind[sc * CT_X + lx] = fluid ? 1 : 0;
    if (fluid) {
      collide_loaded(
          L, cur, x, y, fl, [&](float r, float& Fx, float& Fy) { tile_force<float, PSEUDO>(L, stencils, g, r, Fx, Fy); },
          inner);
      // fl holds the post-collision populations: direction i lands at (lx + ex(i), row + ey(i))
      auto at = [&](int i, int slot, int col) -> float& { return ring[(i * SW_R + slot) * SW_W + col]; };
      at(0, sc, lx + 1) = fl[0];
      at(1, sc, lx + 2) = fl[1];
      at(2, sp1, lx + 1) = fl[2];
      at(3, sc, lx) = fl[3];
      at(4, sm1, lx + 1) = fl[4];
      at(5, sp1, lx + 2) = fl[5];
      at(6, sp1, lx) = fl[6];
      at(7, sm1, lx) = fl[7];
      at(8, sm1, lx + 2) = fl[8];
    }
    __syncthreads();
    // rows y0 - 1 .. y0 + 6 are complete; thread (lx, ly) forms row y0 - 1 + ly, whose ring row
    // is sm1.  The band's first row, and the row below it, wait for k_rho_sweep_fix.
    const int yd = y - 1;
    if (yd > ya && lx > 0 && lx < CT_X - 1 && rkind[sm1 * CT_X + lx]) {
      float fi[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) fi[i] = ring[(i * SW_R + sm1) * SW_W + lx + 1];
      const float r = density_of(L, fi);
      const int n = yd * L.pitch + x;
      A.rho_next[n] = r;
      L.psip[n] = psi_prime_shifted(L, r);
    }
    if (threadIdx.x < 18 * CT_Y) {
      const int e = threadIdx.x / CT_Y, j = threadIdx.x % CT_Y;
      const int ye = y0 - 1 + j;
      if (ye > ya) {
        int dir, rcol, ecol;
        sweep_edge_entry(e, tx, A.strips, dir, rcol, ecol);
        const int se = (ye - ya + 1) % SW_R;
        A.edge[((long long)dir * 2 * A.strips + ecol) * L.ny + ye] = ring[(dir * SW_R + se) * SW_W + rcol];
      }
    }
  }
}

// What the sweep left: the densities (and psi'(rho) - mu_sat) of the strips' edge columns in
// band-interior rows, from the edge buffer, then those of the bands' first and last rows, from
// the new populations (lattice `cur`).  The same sum as the density pass.
__global__ void __launch_bounds__(NODE_BLOCK) k_rho_sweep_fix(Lattice<float> L, int cur, SweepArgs A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n_edge = 2LL * A.strips * L.ny;
  float fi[9];
  int n;
  if (t < n_edge) {
    const int col = (int)(t / L.ny), y = (int)(t - (long long)col * L.ny);
    const int tr = y / CT_Y;
    int b = (int)((long long)tr * A.bands / A.tile_rows);
    while (b + 1 < A.bands && sweep_band_start(b + 1, A.bands, A.tile_rows) <= tr) ++b;
    if (y == sweep_band_start(b, A.bands, A.tile_rows) * CT_Y || y == sweep_band_start(b + 1, A.bands, A.tile_rows) * CT_Y - 1)
      return;
    const int x = (col >> 1) * CT_X + ((col & 1) ? CT_X - 1 : 0);
    n = y * L.pitch + x;
    if (L.kind[n] != KIND_FLUID) return;
#pragma unroll
    for (int i = 0; i < 9; ++i) fi[i] = A.edge[((long long)i * 2 * A.strips + col) * L.ny + y];
  } else {
    const long long u = t - n_edge;
    if (u >= 2LL * A.bands * L.nx) return;
    const int row = (int)(u / L.nx), x = (int)(u - (long long)row * L.nx);
    const int b = row >> 1;
    const int y = (row & 1) ? sweep_band_start(b + 1, A.bands, A.tile_rows) * CT_Y - 1
                            : sweep_band_start(b, A.bands, A.tile_rows) * CT_Y;
    n = y * L.pitch + x;
    if (L.kind[n] != KIND_FLUID) return;
    const float* __restrict__ f = L.f[cur];
#pragma unroll
    for (int i = 0; i < 9; ++i) fi[i] = f[i * L.plane + n];
  }
  const float r = density_of(L, fi);
  A.rho_next[n] = r;
  L.psip[n] = psi_prime_shifted(L, r);
}

// Boundary links, then the deterministic domain sum of this step's Eq. 18 compensation into
// the per-step ring (two-level reduction, the last block to finish sums the partials).
template <typename real, bool PSEUDO>
__global__ void __launch_bounds__(NODE_BLOCK) k_bc(Lattice<real> L, int cur) {
  __shared__ double red[32];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  double sum = b < L.n_bnodes ? phase_bc<real, 4, PSEUDO>(L, cur, b) : 0.0;
  if (b < L.b_lo || b >= L.b_hi) sum = 0.0;   // a slab's halo nodes belong to its neighbour's sum
  double bt = block_sum(sum, red);
  double total;
  if (finish_reduction(bt, L.partials, L.counter, &total, red)) {
    unsigned long long st = *L.step_ctr;
    L.dM_ring[st % DM_RING] = total;
    L.dM_ring[DM_RING] = total;   // the last step's value, for a read-back without the counter
    *L.step_ctr = st + 1;
  }
}

// Eq. 15 for the first solid layer from the boundary nodes' densities in rho_b (every fluid
// neighbour of a solid node is a boundary node): the sum phase_solid forms, in its order, so
// the first layer can be done before the density plane of the new state is complete.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_solid1_b(Lattice<real> L) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.n_s1) return;
  const uint8_t m = L.s1mask[j];
  real acc = real(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (m & (1u << (i - 1))) acc += real(wgt(i)) * L.rho_b[L.s1nb[8 * j + i - 1]];
  }
  const real rs = acc * L.s1winv[j];
  L.rho[L.s1node[j]] = rs;
  if (L.pseudo && L.eos != EOS_NONE) L.mu[L.s1node[j]] = psi_wall(L, L.s1node[j], rs);
}

// Boundary nodes' densities, left by the boundary phase in rho_b, into the density plane.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_rho_scatter(Lattice<real> L) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < L.n_bnodes) {
    const real r = L.rho_b[b];
    L.rho[L.bnode[b]] = r;
    if (L.psip) L.psip[L.bnode[b]] = psi_prime_shifted(L, r);
    else if (L.pseudo && L.eos != EOS_NONE) L.mu[L.bnode[b]] = psi_of(L, r);
  }
}

// A binary32 value as binary64, exactly: normal numbers and zeros by rebuilding the bit fields
// (sign; exponent rebiased from 127 to 1023; the 23 fraction bits on top of the 52), on the
// integer units -- GB300's FP64 units are few, and the audit's nine conversions a node would
// compete with its nine additions for them; subnormal, infinite and NaN inputs by the conversion.
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) {
  const unsigned int u = __float_as_uint(v);
  const unsigned int e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u || e == 0xffu) {
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
    return (double)v;
  }
  const unsigned long long bits =
      sign | ((unsigned long long)(e + (1023u - 127u)) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// The sum of a node's nine populations.  FP64: in FP64.  FP32: Knuth's TwoSum carries the
// rounding error of each FP32 addition exactly, and the errors are summed in FP32; the node's sum
// is the FP32 sum plus that error term, both widened to FP64 (the compensated summation of
// Ogita, Rump and Oishi, 2005: within gamma_8^2 sum_i |f_i| ~ (8 u)^2 sum_i |f_i| of the exact
// sum, u = 2^-24, i.e. 2.3e-13 of sum_i |f_i|, against the FP32 state's own 6e-8).  It takes two FP64 additions a node where the
// plain FP64 sum takes nine; GB300's FP64 rate made those the audit's cost.
__device__ __forceinline__ double node_sum(const double (&fl)[9]) {
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) t += fl[i];
  return t;
}
__device__ __forceinline__ double node_sum(const float (&fl)[9]) {
  float p = fl[0], e = 0.f;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const float a = p, b = fl[i];
    p = __fadd_rn(a, b);
    const float bb = __fsub_rn(p, a);
    e = __fadd_rn(e, __fadd_rn(__fsub_rn(a, __fsub_rn(p, bb)), __fsub_rn(b, bb)));
  }
  return to_f64(p) + to_f64(e);
}

// FP64 mass audit: sum over fluid nodes of sum_i (f_i - w_i rho_ref), plus a count of
// non-finite populations.  The host adds n_fluid * rho_ref.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_mass(Lattice<real> L, int cur) {
  __shared__ double red[32];
  __shared__ double red2[32];
  double s = 0.0, bad = 0.0;
  int nbad = 0;
  const real* __restrict__ f = L.f[cur];
  const long long n_lo = (long long)L.own_lo * L.pitch, n_hi = (long long)L.own_hi * L.pitch;
  for (long long n = n_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x; n < n_hi;
       n += (long long)gridDim.x * blockDim.x) {
    if (L.kind[n] != KIND_FLUID) continue;
    real fl[9];
    if (L.aa) {
      load_pops(L, cur, (int)(n % L.pitch), (int)(n / L.pitch), fl);
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) fl[i] = f[i * L.plane + n];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) nbad += isfinite(fl[i]) ? 0 : 1;
    s += node_sum(fl);
  }
  bad = (double)nbad;
  double bs = block_sum(s, red);
  double bb = block_sum(bad, red2);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    L.partials[2 * blockIdx.x] = bs;
    L.partials[2 * blockIdx.x + 1] = bb;
    __threadfence();
    unsigned int prev = atomicAdd(L.counter, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, c = 0.0;
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
    a += ((volatile double*)L.partials)[2 * k];
    c += ((volatile double*)L.partials)[2 * k + 1];
  }
  double ta = block_sum(a, red);
  double tc = block_sum(c, red2);
  if (threadIdx.x == 0) {
    L.scalars[0] = ta;
    L.scalars[1] = tc;
    *L.counter = 0u;
  }
}

// Density and v = u + F/(2 rho) of the current state into dense nx*ny arrays.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_fields(Lattice<real> L, int cur, real* rho_out, real* vx_out,
                                                       real* vy_out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= L.plane) return;
  const int x = (int)(n % L.pitch), y = (int)(n / L.pitch);
  if (x >= L.nx) return;
  const long long d = (long long)y * L.nx + x;
  if (L.kind[n] != KIND_FLUID) {
    rho_out[d] = real(0);
    vx_out[d] = real(0);
    vy_out[d] = real(0);
    return;
  }
  real fl[9];
  load_pops(L, cur, x, y, fl);
  real drho, jx, jy;
  moments(fl, drho, jx, jy);
  const real r = L.rho_ref + drho;
  real Fx, Fy;
  if (L.pseudo) force_at<real, true>(L, x, y, r, Fx, Fy);
  else force_at<real, false>(L, x, y, r, Fx, Fy);
  rho_out[d] = r;
  vx_out[d] = (jx + real(0.5) * Fx) / r;
  vy_out[d] = (jy + real(0.5) * Fy) / r;
}

// One double into page-locked host memory (its device address), in stream order.
__global__ void k_copy8(const double* __restrict__ src, double* dst) { *dst = *src; }
cudaError_t launch_copy8(const double* src, double* dst, cudaStream_t s) {
  k_copy8<<<1, 1, 0, s>>>(src, dst);
  return cudaGetLastError();
}

// Largest speed |v| = |u + F/(2 rho)| over the fluid nodes of the current state, combined into
// *out as FP64 bits (the caller zeroes it): non-negative doubles order like their bit patterns,
// and a NaN, stored as the positive quiet NaN, lies above every number.  The speed is formed in
// FP64 from the velocity k_fields writes, squares and sum rounded in that order.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_max_speed(Lattice<real> L, int cur, unsigned long long* out) {
  unsigned long long b = 0ull;
  const long long n_lo = (long long)L.own_lo * L.pitch, n_hi = (long long)L.own_hi * L.pitch;
  for (long long n = n_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x; n < n_hi;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % L.pitch), y = (int)(n / L.pitch);
    if (x >= L.nx || L.kind[n] != KIND_FLUID) continue;
    real fl[9];
    load_pops(L, cur, x, y, fl);
    real drho, jx, jy;
    moments(fl, drho, jx, jy);
    const real r = L.rho_ref + drho;
    real Fx, Fy;
    if (L.pseudo) force_at<real, true>(L, x, y, r, Fx, Fy);
    else force_at<real, false>(L, x, y, r, Fx, Fy);
    const double vx = (double)((jx + real(0.5) * Fx) / r), vy = (double)((jy + real(0.5) * Fy) / r);
    const double sp = sqrt(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)));
    const unsigned long long bits = sp == sp ? (unsigned long long)__double_as_longlong(sp) : 0x7ff8000000000000ull;
    b = bits > b ? bits : b;
  }
  __shared__ unsigned long long part[NODE_BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
    b = v > b ? v : b;
  }
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NODE_BLOCK / 32; ++w) b = part[w] > b ? part[w] : b;
    atomicMax(out, b);
  }
}

// Density of the nodes (x, y0 + j), j < n, of the current state (NaN at solid nodes), in FP64.
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_column(Lattice<real> L, int cur, int x, int y0, int n, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int node = (y0 + j) * L.pitch + x;
  if (L.kind[node] != KIND_FLUID) {
    out[j] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  real fl[9];
  load_pops(L, cur, x, y0 + j, fl);
  out[j] = (double)density_of(L, fl);
}

// Populations i0 <= i < i1 of the current state as absolute values, population i into the
// dense plane i - i0 of `out` (0 at non-fluid nodes).
template <typename real>
__global__ void k_populations(Lattice<real> L, int cur, real* out, int i0, int i1) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= L.plane) return;
  const int x = (int)(n % L.pitch), y = (int)(n / L.pitch);
  if (x >= L.nx) return;
  const long long d = (long long)y * L.nx + x;
  const long long dn = (long long)L.nx * L.ny;
  const bool fluid = L.kind[n] == KIND_FLUID;
  for (int i = i0; i < i1; ++i)
    out[(i - i0) * dn + d] = fluid ? L.f[cur][pop_index(L, cur, i, x, y)] + real(wgt(i)) * L.rho_ref : real(0);
}

// inverse of k_populations: fluid nodes of lattice `cur` from 9 row-major arrays of absolute
// populations (other nodes keep their values)
// (populations i0 <= i < i1, population i from the dense plane i - i0 of `in`)
template <typename real>
__global__ void k_set_populations(Lattice<real> L, int cur, const real* in, int i0, int i1) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= L.plane) return;
  const int x = (int)(n % L.pitch), y = (int)(n / L.pitch);
  if (x >= L.nx || L.kind[n] != KIND_FLUID) return;
  const long long d = (long long)y * L.nx + x;
  const long long dn = (long long)L.nx * L.ny;
  for (int i = i0; i < i1; ++i) L.f[cur][pop_index(L, cur, i, x, y)] = in[(i - i0) * dn + d] - real(wgt(i)) * L.rho_ref;
}

// Eq. 19 initial state: rho = (rho_g + rho_l)/2 + (rho_g - rho_l)/2 tanh(2(r - r0)/W) around
// the droplet with the largest liquid fraction phi at the node, u = phi u0, f = f^eq.
// Population i of the equilibrium with density r and velocity (ux, uy), in offset form (FP64, then
// rounded to the storage type).
template <typename real>
__device__ __forceinline__ real init_pop(int i, double r, double ux, double uy, double rref) {
  const double usq = 1.5 * (ux * ux + uy * uy);
  const double eu = ex(i) * ux + ey(i) * uy;
  const double feq = wgt(i) * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - usq);
  return (real)(feq - wgt(i) * rref);
}
__device__ __forceinline__ double init_rho(double phi, double rho_g, double rho_l) {
  return 0.5 * (rho_g + rho_l) + 0.5 * (rho_g - rho_l) * (1.0 - 2.0 * phi);
}
// A droplet contributes phi = 0 where 2(r - r0)/W >= 40, i.e. r >= r0 + 20 W: there tanh is 1 to
// far below the last bit of a double, so the node skips the square root and tanh.  Nodes that no
// droplet reaches (phi = 0, u = 0: the gas) all get the same populations, formed once per block.
// An FP32 screen of the far test below, exact where it decides: for node coordinates, drop
// centres and far radii below 2^13 the FP32 d^2 lies within 134 of the exact one (the centre and
// the difference rounded once each, 2^-10 in all; the two squares and their sum), so a node with
// d2f > far^2 (1 + 1e-9) + 256 (that bound rounded to FP32, within 4) is far in the FP64 test
// too.  The rest, and drops out of range (bound +inf), take the FP64 test.
constexpr int INIT_SCREEN_MAX = 32;
constexpr int INIT_SCREEN_COORD = 8192;

// grid (ceil(pitch / NODE_BLOCK), up to INIT_ROW_BLOCKS): one node of a row a thread, rows
// blockIdx.y, blockIdx.y + gridDim.y, ... (the per-block set-up is paid once for all of them)
constexpr int INIT_ROW_BLOCKS = 512;
template <typename real>
__global__ void __launch_bounds__(NODE_BLOCK) k_init(Lattice<real> L, const double* __restrict__ drops, int n_drop,
                                                     double W, double rho_g, double rho_l) {
  __shared__ real gas[9];
  __shared__ real gas_rho;
  __shared__ float3 scr[INIT_SCREEN_MAX];
  const double rref = (double)L.rho_ref;
  if (threadIdx.x < 9) gas[threadIdx.x] = init_pop<real>(threadIdx.x, init_rho(0.0, rho_g, rho_l), 0.0, 0.0, rref);
  if (threadIdx.x == 0) gas_rho = (real)init_rho(0.0, rho_g, rho_l);
  if ((int)threadIdx.x < n_drop && threadIdx.x < INIT_SCREEN_MAX) {
    const double* p = drops + 5 * threadIdx.x;
    const double far = p[2] + 20.0 * W;
    const double lim = (double)INIT_SCREEN_COORD;
    const bool ok = fabs(p[0]) < lim && fabs(p[1]) < lim && far > 0.0 && far < lim;
    scr[threadIdx.x] = ok ? make_float3((float)p[0], (float)p[1], (float)(far * far * (1.0 + 1e-9) + 256.0))
                          : make_float3(0.f, 0.f, __int_as_float(0x7f800000));
  }
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= L.pitch) return;
  real* f0 = L.f[0];
  real* f1 = L.f[1];
  const int rows = (int)(L.plane / L.pitch);
  for (int y = blockIdx.y; y < rows; y += gridDim.y) {
    const long long n = (long long)y * L.pitch + x;
    if (x >= L.nx || L.kind[n] != KIND_FLUID) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        f0[i * L.plane + n] = real(0);
        if (!L.aa) f1[i * L.plane + n] = real(0);
      }
      continue;
    }
    const int gy = global_row(L, y);
    const bool fast = x < INIT_SCREEN_COORD && gy >= 0 && gy < INIT_SCREEN_COORD;
    double phi = 0.0, u0 = 0.0, v0 = 0.0;
    for (int d = 0; d < n_drop; ++d) {
      if (fast && d < INIT_SCREEN_MAX) {
        const float3 sc = scr[d];
        const float dxf = __fsub_rn((float)x, sc.x), dyf = __fsub_rn((float)gy, sc.y);
        if (__fadd_rn(__fmul_rn(dxf, dxf), __fmul_rn(dyf, dyf)) > sc.z) continue;
      }
      const double* p = drops + 5 * d;
      double dx = x - p[0], dy = gy - p[1];
      const double d2 = dx * dx + dy * dy;
      const double far = p[2] + 20.0 * W;
      if (far > 0.0 && d2 >= far * far * (1.0 + 1e-9)) continue;
      double rr = sqrt(d2);
      double ph = 0.5 - 0.5 * tanh(2.0 * (rr - p[2]) / W);
      if (ph > phi) { phi = ph; u0 = p[3]; v0 = p[4]; }
    }
    if (phi == 0.0) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        f0[i * L.plane + n] = gas[i];
        if (!L.aa) f1[i * L.plane + n] = real(0);
      }
      L.rho[n] = gas_rho;
      continue;
    }
    const double r = init_rho(phi, rho_g, rho_l);
    const double ux = u0 * phi, uy = v0 * phi;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      f0[i * L.plane + n] = init_pop<real>(i, r, ux, uy, rref);
      if (!L.aa) f1[i * L.plane + n] = real(0);
    }
    L.rho[n] = (real)r;
  }
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
static inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }
template <typename real>
static inline dim3 node_grid(const Lattice<real>& L) {
  return dim3((unsigned)((L.nx + TILE_X - 1) / TILE_X), (unsigned)((L.ny + TILE_Y - 1) / TILE_Y));
}
static inline dim3 node_block() { return dim3(TILE_X, TILE_Y); }
template <typename real>
static inline dim3 collide_grid(const Lattice<real>& L) {
  return dim3((unsigned)((L.nx + CT_X - 1) / CT_X), (unsigned)((L.ny + CT_Y - 1) / CT_Y));
}
template <typename real>
static inline dim3 rho_grid(const Lattice<real>& L) {
  const int nv = (L.nx + Vec16<real>::V - 1) / Vec16<real>::V;
  return dim3((unsigned)((nv + NODE_BLOCK - 1) / NODE_BLOCK), (unsigned)L.ny);
}

// the chemical-potential (or psi) pass, the collide and the boundary kernel of the lattice's
// force model
// the collide kernel of the lattice: the TMA-pipelined one where its descriptors match the
// planes of this step (the reverse sweep's recomputation points elsewhere), else the plain one
template <typename real>
static inline const CollideTma* tma_for(const Lattice<real>& L, int cur) {
  if constexpr (sizeof(real) == 4) {
    const CollideTma* T = static_cast<const CollideTma*>(L.tma);
    if (T && L.f[cur] == T->f_ptr[cur] && (L.mu == T->mu_ptr[0] || L.mu == T->mu_ptr[1]) &&
        (L.rho == T->rho_ptr[0] || L.rho == T->rho_ptr[1]))
      return T;
  }
  return nullptr;
}

// the chemical-potential (or psi) pass; with psi' from the density pass, the vector kernel
// the step forms mu with the next state's density (k_rho_mu_tile) instead of a separate pass
template <typename real>
static inline bool fused_mu(const Lattice<real>& L) {
  return sizeof(real) == 4 && L.mu_kernel == 3 && !L.pseudo && L.eos != EOS_NONE && L.psip != nullptr;
}

template <typename real>
static inline void launch_mu(const Lattice<real>& L, cudaStream_t s) {
  if (L.eos == EOS_NONE) return;
  if (L.pseudo) k_psi<real><<<rho_grid(L), NODE_BLOCK, 0, s>>>(L);
  else if (L.psip && L.mu_kernel >= 2 && sizeof(real) == 4) {
    if constexpr (sizeof(real) == 4) {
      const unsigned gx = (unsigned)((L.nx + 4 * MU_BLOCK - 1) / (4 * MU_BLOCK));
      k_mu_sweep<<<dim3(gx, (unsigned)((L.ny + MU_ROWS - 1) / MU_ROWS)), MU_BLOCK, 0, s>>>(L);
    }
  } else if (L.psip && L.mu_kernel != 0) k_mu_vec<real><<<rho_grid(L), NODE_BLOCK, 0, s>>>(L);
  else k_mu<real><<<node_grid(L), node_block(), 0, s>>>(L);
}
static inline CollideMaps maps_for(const CollideTma* T, const Lattice<float>& L, int cur, bool pull = false) {
  CollideMaps M;
  M.f = pull ? T->f_pull : T->f[cur];
  M.rho = T->rho[L.rho == T->rho_ptr[1] ? 1 : 0];
  M.mu = T->mu[L.mu == T->mu_ptr[1] ? 1 : 0];
  return M;
}
// does this step form the next density in the collide kernel (column sweeps)?
template <typename real>
static inline bool sweep_ready(const Lattice<real>& L, int cur) {
  if constexpr (sizeof(real) == 4) {
    const CollideTma* T = tma_for(L, cur);
    return L.sweep && T && T->edge && !L.pseudo && L.eos != EOS_NONE && L.psip && L.mu_kernel != 3 &&
           L.nx % CT_X == 0 && L.ny % CT_Y == 0;
  }
  return false;
}
// the sweep's work: strips of 32 columns by bands of tile rows, one block each, as many bands
// as fill the device once
static inline SweepArgs sweep_args(const Lattice<float>& L, const CollideTma* T, float* rho_next) {
  SweepArgs A;
  A.rho_next = rho_next;
  A.edge = T->edge;
  A.strips = L.nx / CT_X;
  A.tile_rows = L.ny / CT_Y;
  const int b = T->sweep_blocks / A.strips;
  A.bands = b < 1 ? 1 : (b > A.tile_rows ? A.tile_rows : b);
  return A;
}
// the density pass of the state held as lattice cur (16-byte rows, or one node a thread where
// the AA order shifts the slots)
template <typename real>
static inline void launch_density(const Lattice<real>& L, int cur, cudaStream_t s) {
  if (L.aa && cur == 1) k_rho_pull<real><<<node_grid(L), node_block(), 0, s>>>(L, cur);
  else k_rho_vec<real><<<rho_grid(L), NODE_BLOCK, 0, s>>>(L, cur);
}
// AA order: the boundary nodes' pre-collision moments, before the collide overwrites them
template <typename real>
static inline void launch_bmom(const Lattice<real>& L, int cur, cudaStream_t s) {
  if (L.aa && L.n_bnodes > 0) k_bmom<real><<<grid_for(L.n_bnodes, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, cur);
}
template <typename real>
static inline void launch_collide(const Lattice<real>& L, int cur, cudaStream_t s) {
  if (L.aa && cur == 1) {
    // the second step of the AA order pulls along shifted rows: the TMA-pipelined kernel with
    // the pull box, or the plain one
    if constexpr (sizeof(real) == 4) {
      const CollideTma* T = tma_for(L, cur);
      if (T && T->pull_ok) {
        const CollideMaps M = maps_for(T, L, cur, true);
        const int tiles_x = (L.nx + CT_X - 1) / CT_X;
        const int tiles = tiles_x * ((L.ny + CT_Y - 1) / CT_Y);
        const int P = L.pseudo ? 1 : 0;
        const int grid = tiles < T->blocks_pull[P] ? tiles : T->blocks_pull[P];
        const size_t smem = collide_smem_bytes(L.pseudo, false, 2);
        const SweepArgs none{};
        if (L.pseudo) k_collide_tma<true, false, 2><<<grid, NODE_BLOCK, smem, s>>>(L, cur, M, tiles_x, tiles, none);
        else k_collide_tma<false, false, 2><<<grid, NODE_BLOCK, smem, s>>>(L, cur, M, tiles_x, tiles, none);
        return;
      }
    }
    if (L.pseudo) k_collide<real, true, 2><<<collide_grid(L), NODE_BLOCK, 0, s>>>(L, cur);
    else k_collide<real, false, 2><<<collide_grid(L), NODE_BLOCK, 0, s>>>(L, cur);
    return;
  }
  if constexpr (sizeof(real) == 4) {
    if (const CollideTma* T = tma_for(L, cur)) {
      const CollideMaps M = maps_for(T, L, cur);
      const int tiles_x = (L.nx + CT_X - 1) / CT_X;
      const int tiles = tiles_x * ((L.ny + CT_Y - 1) / CT_Y);
      const int P = L.pseudo ? 1 : 0;
      const int blocks = L.aa ? T->blocks_inplace[P] : T->blocks[P];
      const int grid = tiles < blocks ? tiles : blocks;
      const size_t smem = collide_smem_bytes(L.pseudo, false);
      const SweepArgs none{};
      if (L.aa) {
        if (L.pseudo) k_collide_tma<true, false, 1><<<grid, NODE_BLOCK, smem, s>>>(L, cur, M, tiles_x, tiles, none);
        else k_collide_tma<false, false, 1><<<grid, NODE_BLOCK, smem, s>>>(L, cur, M, tiles_x, tiles, none);
      } else if (L.pseudo) {
        k_collide_tma<true, false><<<grid, NODE_BLOCK, smem, s>>>(L, cur, M, tiles_x, tiles, none);
      } else {
        k_collide_tma<false, false><<<grid, NODE_BLOCK, smem, s>>>(L, cur, M, tiles_x, tiles, none);
      }
      return;
    }
  }
  if (L.aa) {
    if (L.pseudo) k_collide<real, true, 1><<<collide_grid(L), NODE_BLOCK, 0, s>>>(L, cur);
    else k_collide<real, false, 1><<<collide_grid(L), NODE_BLOCK, 0, s>>>(L, cur);
  } else if (L.pseudo) {
    k_collide<real, true><<<collide_grid(L), NODE_BLOCK, 0, s>>>(L, cur);
  } else {
    k_collide<real, false><<<collide_grid(L), NODE_BLOCK, 0, s>>>(L, cur);
  }
}
// collide (column sweeps) of lattice cur into cur ^ 1, the next density into rho_next; then the
// densities the sweep left
template <typename real>
static inline void launch_collide_sweep(const Lattice<real>& L, int cur, real* rho_next, cudaStream_t s) {
  if constexpr (sizeof(real) == 4) {
    const CollideTma* T = tma_for(L, cur);
    const SweepArgs A = sweep_args(L, T, rho_next);
    k_collide_tma<false, true><<<A.strips * A.bands, NODE_BLOCK, collide_smem_bytes(false, true), s>>>(
        L, cur, maps_for(T, L, cur), 0, 0, A);
  }
}
template <typename real>
static inline void launch_sweep_fix(const Lattice<real>& Lt, const Lattice<real>& Ln, int cur, cudaStream_t s) {
  if constexpr (sizeof(real) == 4) {
    const SweepArgs A = sweep_args(Lt, tma_for(Lt, cur), Ln.rho);
    const long long n = 2LL * A.strips * Ln.ny + 2LL * A.bands * Ln.nx;
    k_rho_sweep_fix<<<grid_for(n, NODE_BLOCK), NODE_BLOCK, 0, s>>>(Ln, cur ^ 1, A);
  }
}
template <typename real>
static inline void launch_bc(const Lattice<real>& L, int cur, cudaStream_t s) {
  const unsigned gb = grid_for(L.n_bnodes, NODE_BLOCK);
  if (L.pseudo) k_bc<real, true><<<gb > 0 ? gb : 1, NODE_BLOCK, 0, s>>>(L, cur);
  else k_bc<real, false><<<gb > 0 ? gb : 1, NODE_BLOCK, 0, s>>>(L, cur);
}

// ---- descriptors of the TMA-pipelined collide kernel
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

bool collide_tma_setup(CollideTma* T, const Lattice<float>& L, const void* rho0, const void* rho1, const void* mu1,
                       void* edge, char* err) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) {
    std::snprintf(err, 256, "the CUDA driver's tensor-map encoder is not available");
    return false;
  }
  const cuuint32_t unit[3] = {1, 1, 1};
  auto fail_enc = [&](const char* what, CUresult r) {
    std::snprintf(err, 256, "tensor map of %s: error %d", what, (int)r);
    return false;
  };
  for (int c = 0; c < 2; ++c) {
    // populations: x (contiguous, the padded row), y (rows), plane (the nine directions)
    const cuuint64_t dim[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.ny, 9};
    const cuuint64_t stride[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4};
    const cuuint32_t box[3] = {CT_X, CT_Y, 9};
    CUresult r = enc(&T->f[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)L.f[c], dim, stride, box, unit,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail_enc("the populations", r);
    T->f_ptr[c] = L.f[c];
  }
  {
    // one lattice in AA order: the pull box of its second step
    const cuuint64_t dim[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.ny, 9};
    const cuuint64_t stride[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4};
    const cuuint32_t box[3] = {TMA_PX, TMA_PY, 9};
    T->pull_ok = L.aa && enc(&T->f_pull, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)L.f[0], dim, stride, box, unit,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  auto plane = [&](CUtensorMap* m, const void* base, CUtensorMapDataType type, int esize, cuuint32_t bx, cuuint32_t by) {
    const cuuint64_t dim[2] = {(cuuint64_t)L.pitch, (cuuint64_t)L.ny};
    const cuuint64_t stride[1] = {(cuuint64_t)L.pitch * esize};
    const cuuint32_t box[2] = {bx, by};
    return enc(m, type, 2, const_cast<void*>(base), dim, stride, box, unit, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  };
  const CUtensorMapDataType F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r;
  if ((r = plane(&T->rho[0], rho0, F32, 4, TMA_HX, TMA_MY)) != CUDA_SUCCESS) return fail_enc("density plane 0", r);
  if ((r = plane(&T->rho[1], rho1, F32, 4, TMA_HX, TMA_MY)) != CUDA_SUCCESS) return fail_enc("density plane 1", r);
  if ((r = plane(&T->mu[0], L.mu, F32, 4, TMA_HX, TMA_MY)) != CUDA_SUCCESS) return fail_enc("the mu plane", r);
  if ((r = plane(&T->mu[1], mu1, F32, 4, TMA_HX, TMA_MY)) != CUDA_SUCCESS) return fail_enc("the second psi plane", r);
  T->rho_ptr[0] = rho0;
  T->rho_ptr[1] = rho1;
  T->mu_ptr[0] = L.mu;
  T->mu_ptr[1] = mu1;
  // persistent grids: every block that fits on the device at once
  int dev = 0, sms = 0, b0 = 0, b1 = 0, b2 = 0, p0 = 0, p1 = 0, i0 = 0, i1 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_collide_tma<false, false>, NODE_BLOCK,
                                                    collide_smem_bytes(false, false)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_collide_tma<true, false>, NODE_BLOCK,
                                                    collide_smem_bytes(true, false)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_collide_tma<false, true>, NODE_BLOCK,
                                                    collide_smem_bytes(false, true)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p0, k_collide_tma<false, false, 2>, NODE_BLOCK,
                                                    collide_smem_bytes(false, false, 2)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_collide_tma<true, false, 2>, NODE_BLOCK,
                                                    collide_smem_bytes(true, false, 2)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&i0, k_collide_tma<false, false, 1>, NODE_BLOCK,
                                                    collide_smem_bytes(false, false, 1)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&i1, k_collide_tma<true, false, 1>, NODE_BLOCK,
                                                    collide_smem_bytes(true, false, 1)) != cudaSuccess) {
    (void)cudaGetLastError();
    std::snprintf(err, 256, "occupancy query failed");
    return false;
  }
  T->blocks[0] = (b0 > 0 ? b0 : 1) * sms;
  T->blocks[1] = (b1 > 0 ? b1 : 1) * sms;
  T->sweep_blocks = (b2 > 0 ? b2 : 1) * sms;
  T->blocks_pull[0] = (p0 > 0 ? p0 : 1) * sms;
  T->blocks_pull[1] = (p1 > 0 ? p1 : 1) * sms;
  T->blocks_inplace[0] = (i0 > 0 ? i0 : 1) * sms;
  T->blocks_inplace[1] = (i1 > 0 ? i1 : 1) * sms;
  T->edge = static_cast<float*>(edge);
  return true;
}

template <typename real>
cudaError_t launch_step(const Lattice<real>& L, int cur, cudaStream_t s) {
  launch_density(L, cur, s);
  if (L.n_s1 > 0) k_solid<real><<<grid_for(L.n_s1, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, 1);
  if (L.n_s2 > 0) k_solid<real><<<grid_for(L.n_s2, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, 2);
  launch_mu(L, s);
  launch_bmom(L, cur, s);
  launch_collide(L, cur, s);
  launch_bc(L, cur, s);
  return cudaGetLastError();
}

// One step whose boundary phase overlaps the density pass of the next step.  Lt describes
// step t (rho = the density plane of lattice cur, holding its fluid AND solid-layer densities;
// rho_b set), Ln the next state (rho = the other density plane).  After the collide the work
// forks.  On s: k_bc, which completes the boundary nodes' populations and leaves their
// densities in rho_b; then the two solid layers of the next state (the first from rho_b, the
// second from the first).  On s2: the density of every fluid node of lattice cur^1 -- final
// everywhere but at boundary nodes.  After the join k_rho_scatter puts the boundary densities
// in place.  The values are those of launch_step; only the order of independent work differs.
template <typename real>
cudaError_t launch_step_overlap(const Lattice<real>& Lt, const Lattice<real>& Ln, int cur, cudaStream_t s,
                                cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join) {
  const Lattice<real>& L = Lt;
  // the fused pass left this state's mu at the end of the previous step; psi (pseudopotential
  // force): the previous step's density pass, scatter and layers
  const bool fused = fused_mu(L);
  const bool sweep = sweep_ready(L, cur);
  cudaError_t e;
  const bool bmom = L.aa && L.n_bnodes > 0;
  if (bmom) {
    // one lattice: the boundary nodes' moments are saved on s2 while mu is formed on s
    e = cudaEventRecord(fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, fork, 0);
    if (e != cudaSuccess) return e;
    launch_bmom(L, cur, s2);
    e = cudaEventRecord(join, s2);
    if (e != cudaSuccess) return e;
  }
  if (!L.pseudo && !fused) launch_mu(L, s);
  if (bmom && (e = cudaStreamWaitEvent(s, join, 0)) != cudaSuccess) return e;
  if (sweep) launch_collide_sweep(L, cur, Ln.rho, s);
  else launch_collide(L, cur, s);
  e = cudaEventRecord(fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, fork, 0);
  if (e != cudaSuccess) return e;
  const unsigned gb = grid_for(L.n_bnodes, NODE_BLOCK);
  launch_bc(L, cur, s);
  if (Ln.n_s1 > 0) k_solid1_b<real><<<grid_for(Ln.n_s1, NODE_BLOCK), NODE_BLOCK, 0, s>>>(Ln);
  if (Ln.n_s2 > 0) k_solid<real><<<grid_for(Ln.n_s2, NODE_BLOCK), NODE_BLOCK, 0, s>>>(Ln, 2);
  if (sweep) {
    launch_sweep_fix(L, Ln, cur, s2);
  } else if (fused) {
    if constexpr (sizeof(real) == 4)
      k_rho_mu_tile<<<dim3((unsigned)((Ln.nx + RM_W - 1) / RM_W), (unsigned)((Ln.ny + RM_H - 1) / RM_H)), NODE_BLOCK, 0,
                      s2>>>(Ln, cur ^ 1);
  } else {
    launch_density(Ln, cur ^ 1, s2);
  }
  e = cudaEventRecord(join, s2);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join, 0);
  if (e != cudaSuccess) return e;
  if (L.n_bnodes > 0) k_rho_scatter<real><<<gb, NODE_BLOCK, 0, s>>>(Ln);
  if (fused && Ln.n_near > 0) k_mu_near<real><<<grid_for(Ln.n_near, NODE_BLOCK), NODE_BLOCK, 0, s>>>(Ln);
  return cudaGetLastError();
}

template <typename real>
int launches_per_step_overlap(const Lattice<real>& L) {
  return launches_per_step(L) + (L.n_bnodes > 0) - (L.pseudo && L.eos != EOS_NONE) - (fused_mu(L) ? 1 : 0) +
         (fused_mu(L) && L.n_near > 0 ? 1 : 0) + (L.aa && L.n_bnodes > 0 ? 1 : 0);
}

// one phase of a step: 0 density, 1 solid layers, 2 chemical potential, 3 force+collide+stream,
// 4 boundary links
template <typename real>
cudaError_t launch_phase(const Lattice<real>& L, int cur, int phase, cudaStream_t s) {
  switch (phase) {
    case 0: launch_density(L, cur, s); break;
    case 1:
      if (L.n_s1 > 0) k_solid<real><<<grid_for(L.n_s1, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, 1);
      if (L.n_s2 > 0) k_solid<real><<<grid_for(L.n_s2, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, 2);
      break;
    case 2: launch_mu(L, s); break;
    case 3:
      launch_bmom(L, cur, s);
      launch_collide(L, cur, s);
      break;
    default: launch_bc(L, cur, s);
  }
  return cudaGetLastError();
}

// The phases of a step whose collide kernel sweeps (step_sweeps), one after another for the
// per-phase timing, in their order: 2 chemical potential, 3 force + collide + stream + most of
// the next density, 4 boundary links, 1 the next state's solid layers, 0 the densities the
// sweep left and the boundary nodes'.  Lt, Ln as for launch_step_overlap.
template <typename real>
cudaError_t launch_phase_sweep(const Lattice<real>& Lt, const Lattice<real>& Ln, int cur, int phase, cudaStream_t s) {
  switch (phase) {
    case 0:
      launch_sweep_fix(Lt, Ln, cur, s);
      if (Lt.n_bnodes > 0) k_rho_scatter<real><<<grid_for(Lt.n_bnodes, NODE_BLOCK), NODE_BLOCK, 0, s>>>(Ln);
      break;
    case 1:
      if (Ln.n_s1 > 0) k_solid1_b<real><<<grid_for(Ln.n_s1, NODE_BLOCK), NODE_BLOCK, 0, s>>>(Ln);
      if (Ln.n_s2 > 0) k_solid<real><<<grid_for(Ln.n_s2, NODE_BLOCK), NODE_BLOCK, 0, s>>>(Ln, 2);
      break;
    case 2: launch_mu(Lt, s); break;
    case 3: launch_collide_sweep(Lt, cur, Ln.rho, s); break;
    default: launch_bc(Lt, cur, s);
  }
  return cudaGetLastError();
}
template <typename real>
bool step_sweeps(const Lattice<real>& L, int cur) {
  return sweep_ready(L, cur);
}

template <typename real>
int launches_per_step(const Lattice<real>& L) {
  return 3 + (L.n_s1 > 0) + (L.n_s2 > 0) + (L.eos != EOS_NONE);
}

// density / solid layers / chemical potential of the current state (for the read-outs)
template <typename real>
cudaError_t launch_macro(const Lattice<real>& L, int cur, cudaStream_t s) {
  launch_density(L, cur, s);
  if (L.n_s1 > 0) k_solid<real><<<grid_for(L.n_s1, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, 1);
  if (L.n_s2 > 0) k_solid<real><<<grid_for(L.n_s2, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, 2);
  launch_mu(L, s);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fields(const Lattice<real>& L, int cur, real* r, real* vx, real* vy, cudaStream_t s) {
  cudaError_t e = launch_macro(L, cur, s);
  if (e != cudaSuccess) return e;
  k_fields<real><<<grid_for(L.plane, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, cur, r, vx, vy);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_max_speed(const Lattice<real>& L, int cur, unsigned long long* out, cudaStream_t s) {
  cudaError_t e = launch_macro(L, cur, s);
  if (e != cudaSuccess) return e;
  const long long blocks = std::min<long long>(grid_for(L.plane, NODE_BLOCK), 152LL * 8);
  k_max_speed<real><<<(unsigned)blocks, NODE_BLOCK, 0, s>>>(L, cur, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_column(const Lattice<real>& L, int cur, int x, int y0, int n, double* out, cudaStream_t s) {
  k_column<real><<<grid_for(n, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, cur, x, y0, n, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_populations(const Lattice<real>& L, int cur, real* out, int i0, int i1, cudaStream_t s) {
  k_populations<real><<<grid_for(L.plane, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, cur, out, i0, i1);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_set_populations(const Lattice<real>& L, int cur, const real* in, int i0, int i1, cudaStream_t s) {
  k_set_populations<real><<<grid_for(L.plane, NODE_BLOCK), NODE_BLOCK, 0, s>>>(L, cur, in, i0, i1);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mass(const Lattice<real>& L, int cur, cudaStream_t s) {
  k_mass<real><<<mass_blocks(), NODE_BLOCK, 0, s>>>(L, cur);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_init(const Lattice<real>& L, const double* drops, int n_drop, double W, double rho_g,
                        double rho_l, cudaStream_t s) {
  const long long rows = L.plane / L.pitch;
  const dim3 grid((unsigned)((L.pitch + NODE_BLOCK - 1) / NODE_BLOCK),
                  (unsigned)(rows < INIT_ROW_BLOCKS ? rows : INIT_ROW_BLOCKS));
  k_init<real><<<grid, NODE_BLOCK, 0, s>>>(L, drops, n_drop, W, rho_g, rho_l);
  return cudaGetLastError();
}

#define LBMGB_INSTANTIATE(real)                                                                          \
  template cudaError_t launch_step<real>(const Lattice<real>&, int, cudaStream_t);                      \
  template int launches_per_step<real>(const Lattice<real>&);                                           \
  template cudaError_t launch_phase<real>(const Lattice<real>&, int, int, cudaStream_t);                \
  template cudaError_t launch_phase_sweep<real>(const Lattice<real>&, const Lattice<real>&, int, int, cudaStream_t); \
  template bool step_sweeps<real>(const Lattice<real>&, int);                                           \
  template cudaError_t launch_macro<real>(const Lattice<real>&, int, cudaStream_t);                     \
  template cudaError_t launch_step_overlap<real>(const Lattice<real>&, const Lattice<real>&, int, cudaStream_t, \
                                                 cudaStream_t, cudaEvent_t, cudaEvent_t);                  \
  template int launches_per_step_overlap<real>(const Lattice<real>&);                                   \
  template cudaError_t launch_fields<real>(const Lattice<real>&, int, real*, real*, real*, cudaStream_t); \
  template cudaError_t launch_populations<real>(const Lattice<real>&, int, real*, int, int, cudaStream_t); \
  template cudaError_t launch_column<real>(const Lattice<real>&, int, int, int, int, double*, cudaStream_t); \
  template cudaError_t launch_max_speed<real>(const Lattice<real>&, int, unsigned long long*, cudaStream_t); \
  template cudaError_t launch_set_populations<real>(const Lattice<real>&, int, const real*, int, int, cudaStream_t); \
  template cudaError_t launch_mass<real>(const Lattice<real>&, int, cudaStream_t);                      \
  template cudaError_t launch_init<real>(const Lattice<real>&, const double*, int, double, double,      \
                                         double, cudaStream_t);
LBMGB_INSTANTIATE(float)
LBMGB_INSTANTIATE(double)

}  // namespace lbmgb
