// Per-node (and per-list-entry) bodies of the phases of one time step, shared by the
// single-lattice kernels (lbm_step.cu) and the batched persistent kernel (lbm_batch.cu), so
// that both run the same arithmetic.
//
// Streaming pushes every population, including those leaving a fluid node towards a solid
// node: they land in the solid node's slot of the destination lattice, where the boundary
// phase reads them back as f~_i(x1, t).  Likewise f~_i(x2, t) has streamed into x1 and
// f~_ibar(x1, t) into x2, so the boundary phase needs no copy of the post-collision lattice.
#pragma once
#include "lbm_device.cuh"

namespace lbmgb {

// density of fluid node (x, y) from its 9 offset populations (Sec. 2.1)
template <typename real>
__device__ __forceinline__ void phase_rho(const Lattice<real>& L, int cur, int x, int y) {
  const int n = y * L.pitch + x;
  if (L.kind[n] != KIND_FLUID) return;
  const real* __restrict__ f = L.f[cur];
  real fl[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fl[i] = f[i * L.plane + n];
  L.rho[n] = density_of(L, fl);
}

// Eq. 15: rho(x_s) = sum_i w_i rho(x_s + e_i) s_w / sum_i w_i s_w over the neighbours of the
// previous layer (fluid for layer 1, layer 1 for layer 2); the mask and 1/sum w_i s_w are
// geometry and were computed once.
template <typename real>
__device__ __forceinline__ void phase_solid(const Lattice<real>& L, int layer, int j) {
  const int n = layer == 1 ? L.s1node[j] : L.s2node[j];
  const uint8_t m = layer == 1 ? L.s1mask[j] : L.s2mask[j];
  const real winv = layer == 1 ? L.s1winv[j] : L.s2winv[j];
  const int x = n % L.pitch, y = n / L.pitch;
  real acc = real(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (m & (1u << (i - 1))) acc += real(wgt(i)) * L.rho[node_at(L, x + ex(i), y + ey(i))];
  }
  L.rho[n] = acc * winv;
}

// Eq. 12 in mesh units, shifted by the constant k^2 mu_sat (only gradients of mu enter
// Eq. 9): mu~ = k^2 (psi'(rho) - mu_sat) - kappa^ lap(rho).  Solid layers keep their
// constant wall value.
template <typename real>
__device__ __forceinline__ void phase_mu(const Lattice<real>& L, int x, int y) {
  const int n = y * L.pitch + x;
  if (L.kind[n] != KIND_FLUID) return;
  Stencil s = stencil_at(L, x, y);
  const real r = L.rho[n];
  L.mu[n] = mu_of(L, psi_prime_shifted(L, r), lap4(L.rho, n, s));
}

// ---- one population lattice in AA order (aa set; the state of lattice 1 holds f_i(x) in slot
// opp(i) of x - e_i, pop_index)

// density of fluid node (x, y) of the state in lattice `cur`, read through pop_index, and the
// pointwise part of Eq. 12 (or psi) with it -- the values phase_rho_vec stores
template <typename real>
__device__ __forceinline__ void phase_rho_pull(const Lattice<real>& L, int cur, int x, int y) {
  const int n = y * L.pitch + x;
  if (L.kind[n] != KIND_FLUID) return;
  real fl[9];
  load_pops(L, cur, x, y, fl);
  const real r = density_of(L, fl);
  L.rho[n] = r;
  if (L.psip) L.psip[n] = psi_prime_shifted(L, r);
  else if (L.pseudo && L.eos != EOS_NONE) L.mu[n] = psi_of(L, r);
}

// the pre-collision moments of boundary node b, which the boundary phase needs after the collide
// has overwritten the populations (the sums of `moments`)
template <typename real>
__device__ __forceinline__ void phase_bmom(const Lattice<real>& L, int cur, int b) {
  const int n = L.bnode[b];
  real fl[9];
  load_pops(L, cur, n % L.pitch, n / L.pitch, fl);
  real drho, jx, jy;
  moments(fl, drho, jx, jy);
  L.bmom[3 * b] = drho;
  L.bmom[3 * b + 1] = jx;
  L.bmom[3 * b + 2] = jy;
}

// ---- 16-byte row vectors: V = 16/sizeof(real) consecutive nodes of a row per thread.  Rows
// start on 128-byte boundaries (the pitch), so every vector at a multiple of V is aligned.
template <typename real> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int V = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int V = 2; };

template <typename real>
__device__ __forceinline__ real lane_of(const typename Vec16<real>::type& v, int k);
template <> __device__ __forceinline__ float lane_of<float>(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
template <> __device__ __forceinline__ double lane_of<double>(const double2& v, int k) { return k == 0 ? v.x : v.y; }
template <typename real>
__device__ __forceinline__ typename Vec16<real>::type make_vec(const real (&a)[Vec16<real>::V]);
template <> __device__ __forceinline__ float4 make_vec<float>(const float (&a)[4]) { return make_float4(a[0], a[1], a[2], a[3]); }
template <> __device__ __forceinline__ double2 make_vec<double>(const double (&a)[2]) { return make_double2(a[0], a[1]); }

// Density of the fluid nodes x0 .. x0+V-1 of row y (x0 < nx, a multiple of V) from 16-byte loads
// of lattice `cur` in natural slot order -- the values phase_rho stores -- and, while the density
// is at hand, the pointwise part of Eq. 12 into psip (chemical-potential force) or psi itself into
// mu (pseudopotential force): this pass is bound by its bytes, the chemical-potential pass by its
// instructions.
template <typename real>
__device__ __forceinline__ void phase_rho_vec(const Lattice<real>& L, int cur, int x0, int y) {
  using VT = typename Vec16<real>::type;
  constexpr int V = Vec16<real>::V;
  const int n0 = y * L.pitch + x0;
  const real* __restrict__ f = L.f[cur];
  VT fv[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fv[i] = __ldg(reinterpret_cast<const VT*>(f + i * L.plane + n0));
  bool fluid[V];
  bool all = true;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    fluid[k] = x0 + k < L.nx && L.kind[n0 + k] == KIND_FLUID;
    all &= fluid[k];
  }
  real* second = L.psip ? L.psip : ((L.pseudo && L.eos != EOS_NONE) ? L.mu : nullptr);
  real r[V], p[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    real fl[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fl[i] = lane_of<real>(fv[i], k);
    r[k] = density_of(L, fl);
    p[k] = (!second || !fluid[k]) ? real(0) : (L.psip ? psi_prime_shifted(L, r[k]) : psi_of(L, r[k]));
  }
  if (all) {
    // every node fluid: 16-byte stores (a solid node's slot belongs to the solid-layer kernels,
    // which may be writing it concurrently, so mixed vectors take the scalar path)
    *reinterpret_cast<VT*>(L.rho + n0) = make_vec<real>(r);
    if (second) *reinterpret_cast<VT*>(second + n0) = make_vec<real>(p);
    return;
  }
#pragma unroll
  for (int k = 0; k < V; ++k) {
    if (!fluid[k]) continue;
    L.rho[n0 + k] = r[k];
    if (second) second[n0 + k] = p[k];
  }
}

// Eq. 12 at the fluid nodes x0 .. x0+V-1 of row y (x0 < nx, a multiple of V) with psi' from the
// density pass: the centre row from three 16-byte loads (x0 - V .. x0 + 2V - 1), the four rows
// above and below and psi' from one each, so the 9-point Laplacians of V nodes take 8 vector loads
// instead of 9 V scalar ones.  Where the stencils would wrap around a periodic edge, node by node.
// Same values and the same sums as phase_mu (lap4_of, mu_of).
template <typename real>
__device__ __forceinline__ void phase_mu_vec(const Lattice<real>& L, int x0, int y) {
  using VT = typename Vec16<real>::type;
  constexpr int V = Vec16<real>::V;
  const int n0 = y * L.pitch + x0;
  bool fluid[V];
  bool any = false;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    fluid[k] = x0 + k < L.nx && L.kind[n0 + k] == KIND_FLUID;
    any |= fluid[k];
  }
  if (!any) return;
  // no wrap within two nodes (with walls a fluid row keeps two solid rows below and above it)
  const bool inner = x0 - V >= 0 && x0 + V + 2 <= L.nx && (L.walls || (y >= 2 && y < L.ny - 2));
  if (!inner) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      if (!fluid[k]) continue;
      Stencil st = stencil_at(L, x0 + k, y);
      L.mu[n0 + k] = mu_of(L, L.psip[n0 + k], lap4(L.rho, n0 + k, st));
    }
    return;
  }
  const real* __restrict__ r = L.rho;
  real c[3 * V];   // the centre row, x0 - V .. x0 + 2V - 1
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const VT v = __ldg(reinterpret_cast<const VT*>(r + n0 + (j - 1) * V));
#pragma unroll
    for (int k = 0; k < V; ++k) c[j * V + k] = lane_of<real>(v, k);
  }
  const VT up1 = __ldg(reinterpret_cast<const VT*>(r + n0 + L.pitch));
  const VT dn1 = __ldg(reinterpret_cast<const VT*>(r + n0 - L.pitch));
  const VT up2 = __ldg(reinterpret_cast<const VT*>(r + n0 + 2 * L.pitch));
  const VT dn2 = __ldg(reinterpret_cast<const VT*>(r + n0 - 2 * L.pitch));
  const VT pp = __ldg(reinterpret_cast<const VT*>(L.psip + n0));
#pragma unroll
  for (int k = 0; k < V; ++k) {
    if (!fluid[k]) continue;
    const int i = V + k;
    const real lap = lap4_of(c[i], c[i + 1], c[i - 1], c[i + 2], c[i - 2], lane_of<real>(up1, k), lane_of<real>(dn1, k),
                             lane_of<real>(up2, k), lane_of<real>(dn2, k));
    L.mu[n0 + k] = mu_of(L, lane_of<real>(pp, k), lap);
  }
}

// ---- collide tiles of 32 x 8 nodes with a two-node halo of the stencil fields in shared memory
constexpr int CT_X = 32, CT_Y = 8, CT_H = 2;
constexpr int CT_SX = CT_X + 2 * CT_H, CT_SY = CT_Y + 2 * CT_H;
static_assert(CT_X == 32 && CT_SX - 32 <= 32, "one warp stages a row of the tile and its halo");

// Terms of the force at a node from a staged tile (row stride W, the node at index c): the
// undivided fourth-order differences of mu and rho of Eq. 9 (diff4_of), or the two sums and the
// centre value of the pseudopotential force.  Both collide kernels take them before the
// collision and finish the force with tile_force, so that they evaluate it with the same
// operations as force_at.
template <typename real, bool PSEUDO>
__device__ __forceinline__ void tile_force_terms(const real* sm, const real* sr, int W, int c, real (&g)[4]) {
  if (PSEUDO) {
    pp_sums(sm[c + 1], sm[c + W], sm[c - 1], sm[c - W], sm[c + W + 1], sm[c + W - 1], sm[c - W - 1], sm[c - W + 1],
            g[0], g[1]);
    g[2] = sm[c];
    g[3] = real(0);
  } else {
    g[0] = diff4_of(sm[c + 1], sm[c - 1], sm[c + 2], sm[c - 2]);
    g[1] = diff4_of(sm[c + W], sm[c - W], sm[c + 2 * W], sm[c - 2 * W]);
    g[2] = diff4_of(sr[c + 1], sr[c - 1], sr[c + 2], sr[c - 2]);
    g[3] = diff4_of(sr[c + W], sr[c - W], sr[c + 2 * W], sr[c - 2 * W]);
  }
}
// F = rho g plus the nonideal force from those terms (force_at's operations)
template <typename real, bool PSEUDO>
__device__ __forceinline__ void tile_force(const Lattice<real>& L, bool stencils, const real (&g)[4], real r, real& Fx,
                                           real& Fy) {
  if (!stencils) {
    Fx = r * L.gx;
    Fy = r * L.gy;
    return;
  }
  if (PSEUDO) {
    Fx = force_pp(r, L.gx, g[2], g[0]);
    Fy = force_pp(r, L.gy, g[2], g[1]);
  } else {
    Fx = force_cp(r, L.gx, g[0], g[2]);
    Fy = force_cp(r, L.gy, g[1], g[3]);
  }
}

// The density and chemical potential (or psi) of the 32 x 8 collide tile at (x0, y0) and of a
// two-node halo into shared memory, by all CT_X * CT_Y threads of the block (the caller
// synchronises before reading them): one warp per row where tile and halo lie inside the
// lattice, else element by element with the periodic wrap.
template <typename real, bool PSEUDO>
__device__ __forceinline__ void stage_tile(const Lattice<real>& L, int x0, int y0, real (*s_rho)[CT_SX],
                                           real (*s_mu)[CT_SX]) {
  constexpr int NT = CT_X * CT_Y;
  if (x0 >= CT_H && x0 + CT_X + CT_H <= L.nx && y0 >= CT_H && y0 + CT_Y + CT_H <= L.ny) {
    // tile and halo inside the lattice (block-uniform): one warp per staged row, plain offsets
    const int lane = threadIdx.x & 31, wr = threadIdx.x >> 5;
    const int base = (y0 - CT_H) * L.pitch + (x0 - CT_H);
    for (int r = wr; r < CT_SY; r += NT / 32) {
      const int row = base + r * L.pitch;
      if (!PSEUDO) s_rho[r][lane] = L.rho[row + lane];
      s_mu[r][lane] = L.mu[row + lane];
      if (lane < CT_SX - 32) {
        if (!PSEUDO) s_rho[r][32 + lane] = L.rho[row + 32 + lane];
        s_mu[r][32 + lane] = L.mu[row + 32 + lane];
      }
    }
  } else {
    for (int e = threadIdx.x; e < CT_SX * CT_SY; e += NT) {
      const int ly = e / CT_SX, lx = e - ly * CT_SX;
      const int x = x0 + lx - CT_H, y = y0 + ly - CT_H;
      real r = real(0), m = real(0);
      // a fluid node's stencil reaches x in [-2, nx+1] (wrapped) and, with walls, stays
      // inside the rows; other slots are never read
      if (x <= L.nx + 1 && (L.walls ? (y >= 0 && y < L.ny) : (y <= L.ny + 1))) {
        const int n = node_at(L, x, y);
        if (!PSEUDO) r = L.rho[n];
        m = L.mu[n];
      }
      if (!PSEUDO) s_rho[ly][lx] = r;
      s_mu[ly][lx] = m;
    }
  }
}

// force (Eq. 9) + collision (Eq. 4) with exact-difference forcing (Eq. 13) + push streaming
// (Eq. 5) of fluid node (x, y) into the other lattice.  Force(r, Fx, Fy) evaluates Eq. 9 at
// the node: from the density and chemical-potential planes (force_at), or from a tile of them
// staged in shared memory -- the same values in the same order of operations.
// The second half of the phase, for populations fl already loaded from lattice `cur`.
// inner: the caller knows that no push of this node wraps around a lattice edge (a whole tile
// one node away from every edge), which skips the per-node test; the destinations are the same.
// INPLACE (the first step of the AA order, one lattice): f~_i goes back into the node's own slot
// opp(i) instead of being pushed to x + e_i -- the slot the AA order reads f_i(x + e_i) from.
template <bool INPLACE = false, typename real, typename Force>
__device__ __forceinline__ void collide_loaded(const Lattice<real>& L, int cur, int x, int y, real (&fl)[9],
                                               Force&& force, bool inner = false) {
  const int n = y * L.pitch + x;
  real drho, jx, jy;
  moments(fl, drho, jx, jy);
  const real r = L.rho_ref + drho;
  real Fx, Fy;
  force(r, Fx, Fy);
  collide_node(L, fl, r, drho, jx, jy, Fx, Fy);
  if (INPLACE) {
    // the one lattice is both source and destination; this node alone reads and writes its slots
    real* f = L.f[0];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[opp(i) * L.plane + n] = fl[i];
    return;
  }
  real* __restrict__ fout = L.f[cur ^ 1];
  int xm = x - 1, xp = x + 1, rowc = y * L.pitch, rowm = rowc - L.pitch, rowp = rowc + L.pitch;
  if (!inner && !interior(L, x, y)) {
    xm = wrap_x(L, x - 1);
    xp = wrap_x(L, x + 1);
    rowm = wrap_y(L, y - 1) * L.pitch;
    rowp = wrap_y(L, y + 1) * L.pitch;
  }
  fout[0 * L.plane + n] = fl[0];
  fout[1 * L.plane + rowc + xp] = fl[1];
  fout[2 * L.plane + rowp + x] = fl[2];
  fout[3 * L.plane + rowc + xm] = fl[3];
  fout[4 * L.plane + rowm + x] = fl[4];
  fout[5 * L.plane + rowp + xp] = fl[5];
  fout[6 * L.plane + rowp + xm] = fl[6];
  fout[7 * L.plane + rowm + xm] = fl[7];
  fout[8 * L.plane + rowm + xp] = fl[8];
}

template <typename real, typename Force>
__device__ __forceinline__ void phase_collide_with(const Lattice<real>& L, int cur, int x, int y, Force&& force) {
  const int n = y * L.pitch + x;
  if (L.kind[n] != KIND_FLUID) return;
  const real* __restrict__ fin = L.f[cur];
  real fl[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fl[i] = fin[i * L.plane + n];
  collide_loaded(L, cur, x, y, fl, force);
}

template <typename real>
__device__ __forceinline__ void phase_collide(const Lattice<real>& L, int cur, int x, int y) {
  phase_collide_with(L, cur, x, y, [&](real r, real& Fx, real& Fy) { force_at(L, x, y, r, Fx, Fy); });
}

// The collide of one lattice in AA order: from the natural order (cur 0) each node's own slots
// are read and rewritten in place; from the shifted order (cur 1) f_i(x) is pulled from slot
// opp(i) of x - e_i and f~_i(x) pushed into slot i of x + e_i.  The arithmetic of phase_collide.
template <typename real>
__device__ __forceinline__ void phase_collide_aa(const Lattice<real>& L, int cur, int x, int y) {
  const int n = y * L.pitch + x;
  if (L.kind[n] != KIND_FLUID) return;
  real fl[9];
  load_pops(L, cur, x, y, fl);
  auto force = [&](real r, real& Fx, real& Fy) { force_at(L, x, y, r, Fx, Fy); };
  if (cur == 0) collide_loaded<true>(L, cur, x, y, fl, force);
  else collide_loaded<false>(L, cur, x, y, fl, force);
}

// Boundary node b (one per thread): rebuild (rho, u, F) of step t at x1 from the
// pre-collision lattice and the rho / mu planes (the arithmetic of the collide phase; PSEUDO:
// the pseudopotential force from the psi plane), apply
// Eq. 16 or 17 on each of its links, and add the FP64 sum of Eq. 18 to f_0.  Returns that sum
// (0 for the schemes without compensation).
//
// PREFETCH > 0 (the single-lattice kernel): the data of the node's first PREFETCH links --
// direction, q, x2 flag, then a, b2, c -- are loaded before the node's own state, so that the
// thread waits on two rounds of loads instead of two per link.  Loading early changes nothing:
// no link reads a value an earlier link of the node writes (a link writes f_ibar(x1) only where
// x1 - e_ibar is solid, and then no other link of x1 reads that slot).  PREFETCH = 0 keeps the
// register count low for the batched kernel.  Both produce identical values.
template <typename real>
__device__ __forceinline__ real edm_dir(int i, real r, real ux, real uy, real dux, real duy) {
  switch (i) {
    case 1: return edm_term<real>(1, r, ux, uy, dux, duy);
    case 2: return edm_term<real>(2, r, ux, uy, dux, duy);
    case 3: return edm_term<real>(3, r, ux, uy, dux, duy);
    case 4: return edm_term<real>(4, r, ux, uy, dux, duy);
    case 5: return edm_term<real>(5, r, ux, uy, dux, duy);
    case 6: return edm_term<real>(6, r, ux, uy, dux, duy);
    case 7: return edm_term<real>(7, r, ux, uy, dux, duy);
    default: return edm_term<real>(8, r, ux, uy, dux, duy);
  }
}

template <typename real, int PREFETCH = 0, bool PSEUDO = false>
__device__ __forceinline__ double phase_bc(const Lattice<real>& L, int cur, int b) {
  const int n = L.bnode[b];
  const int x = n % L.pitch, y = n / L.pitch;
  real* fout = L.f[cur ^ 1];
  const int nc = cur ^ 1;   // the state after the collide, in its slot order (pop_index)
  const int l0 = L.bstart[b], l1 = L.bstart[b + 1];
  constexpr int P = PREFETCH > 0 ? PREFETCH : 1;
  int pd[P];
  real pq[P], pa[P], pb[P], pc[P];
  uint8_t pf[P];
  if (PREFETCH > 0) {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      pd[k] = 1;
      if (l0 + k < l1) {
        pd[k] = L.ldir[l0 + k];
        pq[k] = L.lq[l0 + k];
        pf[k] = L.lx2f[l0 + k];
      }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      if (l0 + k < l1) {
        const int i = pd[k];
        pa[k] = fout[pop_index(L, nc, i, x + ex(i), y + ey(i))];
        pb[k] = fout[pop_index(L, nc, i, x, y)];
        pc[k] = fout[pop_index(L, nc, opp(i), x - ex(i), y - ey(i))];
      }
    }
  }
  real drho, jx, jy;
  if (L.aa) {
    // one lattice: the collide has overwritten the node's pre-collision populations; their
    // moments were saved before it (k_bmom, the same sums)
    drho = L.bmom[3 * b];
    jx = L.bmom[3 * b + 1];
    jy = L.bmom[3 * b + 2];
  } else {
    const real* __restrict__ fin = L.f[cur];
    real fl[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fl[i] = fin[i * L.plane + n];
    moments(fl, drho, jx, jy);
  }
  const real r = L.rho_ref + drho;
  real Fx, Fy;
  force_at<real, PSEUDO>(L, x, y, r, Fx, Fy);
  const real inv_r = real(1) / r;
  const real ux = jx * inv_r, uy = jy * inv_r, dux = Fx * inv_r, duy = Fy * inv_r;
  double sum = 0.0;
  for (int l = l0; l < l1; ++l) {
    const int k = l - l0;
    int i;
    real q, a, b2, c;
    int x2f;
    if (PREFETCH > 0 && k < P) {
      // registers indexed by a loop counter: select among the unrolled slots
      i = pd[0]; q = pq[0]; a = pa[0]; b2 = pb[0]; c = pc[0]; x2f = pf[0];
#pragma unroll
      for (int s = 1; s < P; ++s)
        if (k == s) { i = pd[s]; q = pq[s]; a = pa[s]; b2 = pb[s]; c = pc[s]; x2f = pf[s]; }
    } else {
      i = L.ldir[l];
      q = L.lq[l];
      x2f = L.lx2f[l];
      a = fout[pop_index(L, nc, i, x + ex(i), y + ey(i))];
      b2 = fout[pop_index(L, nc, i, x, y)];
      c = fout[pop_index(L, nc, opp(i), x - ex(i), y - ey(i))];
    }
    const int ib = opp(i);
    // F_i(x1, t) of direction i
    const real Fi = edm_dir<real>(i, r, ux, uy, dux, duy);
    const real v = link_rule<real>(L.bc, q, x2f, a, b2, c, Fi);
    fout[pop_index(L, nc, ib, x, y)] = v;
    sum += (double)a - (double)v;
  }
  if (L.bc == BC_PRESENT || L.bc == BC_MIBC) {
    // Eq. 18 on f_0, accumulated in FP64.  The part of the sum that the storage precision
    // cannot hold is carried to the node's next step instead of being dropped, so that the
    // mass stays conserved to FP64 accuracy over any number of steps.
    const double t = (double)fout[n] + sum + L.carry[b];
    const real stored = (real)t;
    L.carry[b] = t - (double)stored;
    fout[n] = stored;
  }
  if (L.rho_b) {
    // the node's populations are final only now: its density for the next step (the sum and
    // order of density_of, as the density pass would take it)
    real g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = fout[pop_index(L, nc, i, x, y)];
    L.rho_b[b] = density_of(L, g);
  }
  return (L.bc == BC_PRESENT || L.bc == BC_MIBC) ? sum : 0.0;
}

}  // namespace lbmgb
