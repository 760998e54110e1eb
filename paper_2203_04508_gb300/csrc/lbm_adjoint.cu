// Reverse (adjoint) mode of one time step, and the droplet objective it is seeded from.
//
// Forward step t (lbm_phases.cuh):  f^t -> rho -> (Eq. 15) solid rho -> (Eq. 12) mu -> (Eq. 9) F
//   -> collision + exact-difference forcing (Eq. 4, 13) -> streaming (Eq. 5) -> cut links
//   (Eqs. 16-17) -> compensation (Eq. 18) -> f^{t+1}.
// Given lambda^{t+1} = dJ/df^{t+1} this file produces lambda^t = dJ/df^t and adds the step's
// share of dJ/d(wall chemical potential) and dJ/d(cylinder centre) (the centre enters only
// through the cut fractions q: |x1 + q e - c|^2 = r^2 gives dq/dc = p / (p . e) with
// p = x1 + q e - c).  The reverse phases run in the opposite order of the forward ones:
//   adj_bc      links and Eq. 18 (per boundary node; the post-collision values a, b2, c the
//               links used are read back from f^{t+1}, where the step left them)
//   adj_collide streaming (pulled) + collision + forcing, per fluid node
//   adj_force   Eq. 9: the force's dependence on mu and rho at the stencil neighbours (gather)
//   adj_mu      Eq. 12: mu's dependence on rho (gather); wall mu -> dJ/d(offset)
//   adj_solid   Eq. 15, second layer then first layer (scatter, atomics)
// The density's share of lambda^t, Lrho (one value per node, the same for all nine
// populations), is not added to the nine planes: lambda^t is kept as (nine planes, Lrho) and the
// next reverse step adds Lrho where it reads lambda.  The forward quantities of step t (rho,
// solid rho, mu) are those the recomputation of the segment stored for that step.
#include "lbm_internal.h"
#include "lbm_phases.cuh"

namespace lbmgb {

constexpr int ADJ_BLOCK = 256;

template <typename real>
__device__ __forceinline__ bool is_field_node(uint8_t k) {
  return k == KIND_FLUID || k == KIND_SOLID1 || k == KIND_SOLID2;
}

// dpsi'/drho = (dp0/drho) / rho (Eq. 7)
template <typename real>
__device__ __forceinline__ real psi_second(const Lattice<real>& L, real r) {
  if (L.eos == EOS_CS) {
    const real eta = L.b * r * real(0.25), om = real(1) - eta;
    const real om2 = om * om;
    const real h1 = (real(1) + eta * (real(4) + eta * (real(4) + eta * (real(-4) + eta)))) / (om2 * om2);
    return L.RT * h1 / r - real(2) * L.a;
  }
  const real x = L.b * r, om = real(1) - x;
  const real D = real(1) + real(2) * x - x * x;
  return L.RT / (r * om * om) - L.aalpha * (real(2) + real(2) * x) / (D * D);
}

// Adjoint of collide_node at one node: lt = dJ/d(post-collision populations); adds
// dJ/d(populations) (direct part) to lf, and dJ/d(delta rho), dJ/dj, dJ/dF to the scalars.
template <typename real>
__device__ __forceinline__ void collide_adjoint(const Lattice<real>& L, real r, real jx, real jy, real Fx, real Fy,
                                                const real (&lt)[9], real (&lf)[9], real& lrho, real& ljx, real& ljy,
                                                real& lFx, real& lFy) {
  const real ir = real(1) / r, ir2 = ir * ir;
  // equilibrium at J' = j + F (the exact-difference term folded in)
  {
    const real Jx = jx + Fx, Jy = jy + Fy, J2 = Jx * Jx + Jy * Jy;
    real lJx = 0, lJy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const real w = real(wgt(i)) * lt[i];
      const real eJ = real(ex(i)) * Jx + real(ey(i)) * Jy;
      lrho += w * (real(1) - real(4.5) * eJ * eJ * ir2 + real(1.5) * J2 * ir2);
      lJx += w * (real(3) * real(ex(i)) + real(9) * eJ * real(ex(i)) * ir - real(3) * Jx * ir);
      lJy += w * (real(3) * real(ey(i)) + real(9) * eJ * real(ey(i)) * ir - real(3) * Jy * ir);
    }
    ljx += lJx;
    ljy += lJy;
    lFx += lJx;
    lFy += lJy;
  }
  if (L.coll == COLL_MRT) {
    // moment-space adjoint of M^-1 (I - S) (M f - m_eq): nu_k = (M lt)_k / D_k (1 - s_k)
    const real s13 = lt[1] + lt[3], s24 = lt[2] + lt[4], s57 = lt[5] + lt[7], s68 = lt[6] + lt[8];
    const real me = (real(-4) * lt[0] - (s13 + s24) + real(2) * (s57 + s68)) * real(1.0 / 36.0) * (real(1) - L.s_e);
    const real mp = (real(4) * lt[0] - real(2) * (s13 + s24) + (s57 + s68)) * real(1.0 / 36.0) * (real(1) - L.s_eps);
    const real mqx = (real(-2) * (lt[1] - lt[3]) + (lt[5] - lt[7]) + (lt[8] - lt[6])) * real(1.0 / 12.0) * (real(1) - L.s_q);
    const real mqy = (real(-2) * (lt[2] - lt[4]) + (lt[5] - lt[7]) + (lt[6] - lt[8])) * real(1.0 / 12.0) * (real(1) - L.s_q);
    const real mxx = (s13 - s24) * real(0.25) * (real(1) - L.s_nu);
    const real mxy = (s57 - s68) * real(0.25) * (real(1) - L.s_nu);
    // M^T nu
    lf[0] += real(-4) * me + real(4) * mp;
    lf[1] += -me - real(2) * mp - real(2) * mqx + mxx;
    lf[2] += -me - real(2) * mp - real(2) * mqy - mxx;
    lf[3] += -me - real(2) * mp + real(2) * mqx + mxx;
    lf[4] += -me - real(2) * mp + real(2) * mqy - mxx;
    lf[5] += real(2) * me + mp + mqx + mqy + mxy;
    lf[6] += real(2) * me + mp - mqx + mqy - mxy;
    lf[7] += real(2) * me + mp - mqx - mqy + mxy;
    lf[8] += real(2) * me + mp + mqx - mqy - mxy;
    // minus the equilibrium moments' dependence on (delta rho, j)
    const real j2 = jx * jx + jy * jy;
    lrho -= me * (real(-2) - real(3) * j2 * ir2) + mp * (real(1) + real(3) * j2 * ir2) -
            mxx * (jx * jx - jy * jy) * ir2 - mxy * jx * jy * ir2;
    ljx -= me * real(6) * jx * ir - mp * real(6) * jx * ir - mqx + mxx * real(2) * jx * ir + mxy * jy * ir;
    ljy -= me * real(6) * jy * ir - mp * real(6) * jy * ir - mqy - mxx * real(2) * jy * ir + mxy * jx * ir;
  } else {
    const real keep = real(1) - L.omega;
    const real j2 = jx * jx + jy * jy;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      lf[i] += keep * lt[i];
      const real w = keep * real(wgt(i)) * lt[i];
      const real ej = real(ex(i)) * jx + real(ey(i)) * jy;
      lrho -= w * (real(1) - real(4.5) * ej * ej * ir2 + real(1.5) * j2 * ir2);
      ljx -= w * (real(3) * real(ex(i)) + real(9) * ej * real(ex(i)) * ir - real(3) * jx * ir);
      ljy -= w * (real(3) * real(ey(i)) + real(9) * ej * real(ey(i)) * ir - real(3) * jy * ir);
    }
  }
}

// populations, moments and force of node n of the stored state (the forward arithmetic)
template <typename real>
__device__ __forceinline__ void node_state(const Lattice<real>& L, int x, int y, real (&f)[9], real& r, real& drho,
                                           real& jx, real& jy, real& Fx, real& Fy) {
  const int n = y * L.pitch + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = L.f[0][i * L.plane + n];
  moments(f, drho, jx, jy);
  r = L.rho_ref + drho;
  force_at(L, x, y, r, Fx, Fy);
}

// ---- adj_bc: one thread per boundary node -------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_bc(Lattice<real> L, AdjBuffers A) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= L.n_bnodes) return;
  const int n = L.bnode[b];
  const int x = n % L.pitch, y = n / L.pitch;
  const real* lin = static_cast<const real*>(A.lam_in);
  const real lrn = static_cast<const real*>(A.Lrho)[n];   // density share of lambda^{t+1} at x1
  real* lbc = static_cast<real*>(A.lam_bc);
  real f[9], r, drho, jx, jy, Fx, Fy;
  node_state(L, x, y, f, r, drho, jx, jy, Fx, Fy);
  // f^{t+1} holds the post-collision values the links used: a = f~_i(x1) parked in the solid
  // node's slot, b2 = f~_i(x2) streamed into x1, c = f~_ibar(x1) streamed into x2 (the link
  // phase overwrites none of them where they are used)
  const real* __restrict__ fn = L.f[1];
  const bool comp = L.bc == BC_PRESENT || L.bc == BC_MIBC;
  const real wF = L.bc == BC_PRESENT ? real(1) : real(0);
  const real l0 = comp ? lin[n] + lrn : real(0);
  const real ir = real(1) / r;
  real lrho = 0, ljx = 0, ljy = 0, lFx = 0, lFy = 0;
  for (int l = L.bstart[b]; l < L.bstart[b + 1]; ++l) {
    const int i = L.ldir[l];
    const int ib = opp(i);
    const real q = L.lq[l];
    const int x2 = node_at(L, x - ex(i), y - ey(i));
    const int xs = node_at(L, x + ex(i), y + ey(i));
    const real a = fn[i * L.plane + xs], c = fn[ib * L.plane + x2];
    const real exi = real(ex(i)), eyi = real(ey(i));
    const real eF = exi * Fx + eyi * Fy, ej = exi * jx + eyi * jy, eJ = ej + eF;
    const real Jx = jx + Fx, Jy = jy + Fy;
    const real Fi = real(wgt(i)) * (real(3) * eF + real(4.5) * (eJ * eJ - ej * ej) * ir -
                                    real(1.5) * ((Jx * Jx + Jy * Jy) - (jx * jx + jy * jy)) * ir);
    const real lR = (lin[ib * L.plane + n] + lrn) - l0;
    real dA = 0, dB = 0, dC = 0, dF = 0, dQ = 0;
    if (L.bc == BC_HBB || (q < real(0.5) && !L.lx2f[l])) {
      dA = 1;
    } else if (q < real(0.5)) {
      const real b2 = fn[i * L.plane + n];
      dA = real(2) * q;
      dB = real(1) - real(2) * q;
      dF = wF * (real(1) - real(2) * q);
      dQ = real(2) * a - real(2) * b2 - real(2) * wF * Fi;
    } else {
      const real i2q = real(1) / (real(2) * q);
      dA = i2q;
      dC = (real(2) * q - real(1)) * i2q;
      dF = wF * dC;
      dQ = (c - a + wF * Fi) * i2q * i2q * real(2);
    }
    atomicAdd(&lbc[i * L.plane + n], dA * lR + l0);
    if (dB != real(0)) atomicAdd(&lbc[i * L.plane + x2], dB * lR);
    if (dC != real(0)) atomicAdd(&lbc[ib * L.plane + n], dC * lR);
    // F_i = w [3 e.F + 4.5 ((e.J')^2 - (e.j)^2)/rho - 1.5 (|J'|^2 - |j|^2)/rho], J' = j + F
    const real lFi = dF * lR;
    if (lFi != real(0)) {
      const real w = real(wgt(i)) * lFi;
      lFx += w * (real(3) * exi + real(9) * eJ * exi * ir - real(3) * Jx * ir);
      lFy += w * (real(3) * eyi + real(9) * eJ * eyi * ir - real(3) * Jy * ir);
      ljx += w * (real(9) * eF * exi - real(3) * Fx) * ir;
      ljy += w * (real(9) * eF * eyi - real(3) * Fy) * ir;
      lrho -= w * (real(4.5) * (eJ * eJ - ej * ej) - real(1.5) * ((Jx * Jx + Jy * Jy) - (jx * jx + jy * jy))) * ir * ir;
    }
    // dJ/dq -> dJ/dc of the cylinder this link cuts
    const int bd = L.body[xs];
    if (bd >= 0 && bd < A.n_cyl && dQ != real(0)) {
      const double gq = (double)dQ * (double)lR;
      const double px = (double)x - L.cyl[4 * bd] + (double)q * ex(i);
      const double py = (double)y - L.cyl[4 * bd + 1] + (double)q * ey(i);
      const double pe = px * ex(i) + py * ey(i);
      atomicAdd(&A.grad[A.n_cyl + 1 + 2 * bd], gq * px / pe);
      atomicAdd(&A.grad[A.n_cyl + 2 + 2 * bd], gq * py / pe);
    }
  }
  real* lrj = static_cast<real*>(A.lrj);
  lrj[n] = lrho;
  lrj[L.plane + n] = ljx;
  lrj[2 * L.plane + n] = ljy;
  real* lF = static_cast<real*>(A.lamF);
  lF[n] = lFx;
  lF[L.plane + n] = lFy;
}

// ---- adj_collide: one thread per fluid node ---------------------------------------------
template <typename real>
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_collide(Lattice<real> L, AdjBuffers A) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= L.nx) return;
  const int n = y * L.pitch + x;
  if (L.kind[n] != KIND_FLUID) return;
  const real* lin = static_cast<const real*>(A.lam_in);
  const real* lrp = static_cast<const real*>(A.Lrho);   // density share of lambda^{t+1}
  real* lout = static_cast<real*>(A.lam_out);
  real* lbc = static_cast<real*>(A.lam_bc);
  real* lrj = static_cast<real*>(A.lrj);
  real* lF = static_cast<real*>(A.lamF);
  real f[9], r, drho, jx, jy, Fx, Fy;
  node_state(L, x, y, f, r, drho, jx, jy, Fx, Fy);
  // adjoint of the post-collision populations: pulled back from where they streamed to
  real lt[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int yy = y + ey(i);
    real v = real(0);
    if (!L.walls || (yy >= 0 && yy < L.ny)) {
      const int m = node_at(L, x + ex(i), yy);
      if (L.kind[m] == KIND_FLUID) v = lin[i * L.plane + m] + lrp[m];
    }
    lt[i] = v;
  }
  real lrho = 0, ljx = 0, ljy = 0, lFx = 0, lFy = 0;
  const uint8_t t = A.bct[n];
  if (t & 1) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      lt[i] += lbc[i * L.plane + n];
      lbc[i * L.plane + n] = real(0);
    }
  }
  if (t & 2) {
    lrho = lrj[n];
    ljx = lrj[L.plane + n];
    ljy = lrj[2 * L.plane + n];
    lFx = lF[n];
    lFy = lF[L.plane + n];
  }
  real lf[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) lf[i] = real(0);
  collide_adjoint(L, r, jx, jy, Fx, Fy, lt, lf, lrho, ljx, ljy, lFx, lFy);
#pragma unroll
  for (int i = 0; i < 9; ++i) lout[i * L.plane + n] = lf[i] + lrho + real(ex(i)) * ljx + real(ey(i)) * ljy;
  lF[n] = lFx;
  lF[L.plane + n] = lFy;
}

// ---- adj_force: Eq. 9, gathered at every node that carries rho or mu ------------------------
template <typename real>
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_force(Lattice<real> L, AdjBuffers A) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= L.nx) return;
  const int n = y * L.pitch + x;
  const uint8_t k = L.kind[n];
  if (!is_field_node<real>(k)) return;
  const real* lF = static_cast<const real*>(A.lamF);
  const real* lFy = lF + L.plane;
  real* Lmu = static_cast<real*>(A.Lmu);
  real* Lrho = static_cast<real*>(A.Lrho);
  real lm = 0, lr = 0;
  if (L.eos != EOS_NONE) {
    // gradient coefficients c_{+1} = 8/12, c_{+2} = -1/12, c_{-d} = -c_d; the neighbour m - d
    // sees this node at offset +d.  Only fluid neighbours carry a force (and so dJ/dF); the
    // density plane holds no value at deep solid nodes, so they are skipped, not multiplied
    // by zero.
    const real c1 = real(8.0 / 12.0), c2 = real(-1.0 / 12.0), cs2 = real(1.0 / 3.0);
    const int dd[4] = {1, -1, 2, -2};
    const real cc[4] = {c1, -c1, c2, -c2};
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      const int yy = y - dd[k2];
      if (!L.walls || (yy >= 0 && yy < L.ny)) {
        const int m = node_at(L, x, yy);
        if (L.kind[m] == KIND_FLUID) {
          const real ly = lFy[m];
          lm -= cc[k2] * (L.rho[m] * ly);
          lr += cs2 * cc[k2] * ly;
        }
      }
      const int mx = node_at(L, x - dd[k2], y);
      if (L.kind[mx] == KIND_FLUID) {
        const real lx = lF[mx];
        lm -= cc[k2] * (L.rho[mx] * lx);
        lr += cs2 * cc[k2] * lx;
      }
    }
  }
  if (k == KIND_FLUID) {
    real gmx = 0, gmy = 0;
    if (L.eos != EOS_NONE) {
      Stencil s = stencil_at(L, x, y);
      grad4(L.mu, s, gmx, gmy);
    }
    lr += lF[n] * (L.gx - gmx) + lFy[n] * (L.gy - gmy);
  }
  Lmu[n] = lm;
  Lrho[n] = lr;
}

// ---- adj_mu: Eq. 12 gathered; wall chemical potential -> dJ/d(offset) ------------------------
template <typename real>
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_mu(Lattice<real> L, AdjBuffers A) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= L.nx) return;
  const int n = y * L.pitch + x;
  const uint8_t k = L.kind[n];
  if (!is_field_node<real>(k) || L.eos == EOS_NONE) return;
  const real* Lmu = static_cast<const real*>(A.Lmu);
  real* Lrho = static_cast<real*>(A.Lrho);
  // mu_m = k^2 psi'(rho_m) - kappa sum_d l_d rho_{m+d}; l_0 = -60/12 (both axes), l_{+-1} =
  // 16/12, l_{+-2} = -1/12; only fluid m carry this dependence
  real acc = 0;
  const int dd[4] = {1, -1, 2, -2};
  const real ll[4] = {real(16.0 / 12.0), real(16.0 / 12.0), real(-1.0 / 12.0), real(-1.0 / 12.0)};
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    const int yy = y - dd[k2];
    if (!L.walls || (yy >= 0 && yy < L.ny)) {
      const int m = node_at(L, x, yy);
      if (L.kind[m] == KIND_FLUID) acc += ll[k2] * Lmu[m];
    }
    const int mx = node_at(L, x - dd[k2], y);
    if (L.kind[mx] == KIND_FLUID) acc += ll[k2] * Lmu[mx];
  }
  real lr = Lrho[n] - L.kappa * acc;
  if (k == KIND_FLUID) {
    lr += -L.kappa * real(-60.0 / 12.0) * Lmu[n] + L.k2 * psi_second(L, L.rho[n]) * Lmu[n];
  } else {
    const int bd = L.body[n];
    atomicAdd(&A.grad[bd >= 0 && bd < A.n_cyl ? bd : A.n_cyl], (double)Lmu[n]);
  }
  Lrho[n] = lr;
}

// ---- adj_solid: Eq. 15 in reverse (second layer, then first) -------------------------------
template <typename real>
__global__ void __launch_bounds__(ADJ_BLOCK) k_adj_solid(Lattice<real> L, AdjBuffers A, int layer) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (layer == 1 ? L.n_s1 : L.n_s2)) return;
  const int n = layer == 1 ? L.s1node[j] : L.s2node[j];
  const uint8_t m = layer == 1 ? L.s1mask[j] : L.s2mask[j];
  const real winv = layer == 1 ? L.s1winv[j] : L.s2winv[j];
  real* Lrho = static_cast<real*>(A.Lrho);
  const real v = Lrho[n] * winv;
  const int x = n % L.pitch, y = n / L.pitch;
#pragma unroll
  for (int i = 1; i < 9; ++i)
    if (m & (1u << (i - 1))) atomicAdd(&Lrho[node_at(L, x + ex(i), y + ey(i))], real(wgt(i)) * v);
}

// ---- set-up, objective, seeds ------------------------------------------------------------
// bct bit 0: node may receive boundary contributions to its post-collision adjoint (x1 or x2 of
// a cut link); bit 1: boundary node (local moment and force adjoints from its links)
template <typename real>
__global__ void k_adj_flags_x2(Lattice<real> L, uint8_t* bct) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= L.n_bnodes) return;
  const int n = L.bnode[b];
  const int x = n % L.pitch, y = n / L.pitch;
  for (int l = L.bstart[b]; l < L.bstart[b + 1]; ++l) {
    const int i = L.ldir[l];
    if (L.lx2f[l]) bct[node_at(L, x - ex(i), y - ey(i))] = 1;
  }
}

template <typename real>
__global__ void k_adj_flags_x1(Lattice<real> L, uint8_t* bct) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= L.n_bnodes) return;
  bct[L.bnode[b]] = 3;
}

// touch[n] = 1 at fluid nodes with a cut link into body `body`
template <typename real>
__global__ void k_touch(Lattice<real> L, uint8_t* touch, int body) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= L.n_bnodes) return;
  const int n = L.bnode[b];
  const int x = n % L.pitch, y = n / L.pitch;
  uint8_t t = 0;
  for (int l = L.bstart[b]; l < L.bstart[b + 1]; ++l) {
    const int i = L.ldir[l];
    if (L.body[node_at(L, x + ex(i), y + ey(i))] == body) t = 1;
  }
  touch[n] = t;
}

// Sums of the droplet objective over the fluid nodes of lattice `cur`, one set per block
// (red[4 b + k]; the host adds the blocks in order, so the result does not depend on timing):
//   k = 0: sum (rho - rho_g), 1: sum (rho - rho_g) y,
//   2: sum over touching nodes of (rho - rho_g)/(rho_l - rho_g), 3: their number.
template <typename real>
__global__ void k_objective_sums(Lattice<real> L, int cur, const uint8_t* touch, double* red, double rg, double rl) {
  __shared__ double sm[32];
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < L.plane; n += gridDim.x * blockDim.x) {
    if (L.kind[n] != KIND_FLUID) continue;
    real fl[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fl[i] = L.f[cur][i * L.plane + n];
    const double r = (double)L.rho_ref + (double)density_sum(fl);
    const double y = (double)(n / L.pitch);
    s0 += r - rg;
    s1 += (r - rg) * y;
    if (touch[n]) {
      s2 += (r - rg) / (rl - rg);
      s3 += 1.0;
    }
  }
  double* out = red + 4 * blockIdx.x;
  double t;
  t = block_sum(s0, sm); if (threadIdx.x == 0) out[0] = t;
  t = block_sum(s1, sm); if (threadIdx.x == 0) out[1] = t;
  t = block_sum(s2, sm); if (threadIdx.x == 0) out[2] = t;
  t = block_sum(s3, sm); if (threadIdx.x == 0) out[3] = t;
}

// dJ/drho of the objective at every node (row-major nx x ny; zero off the fluid)
template <typename real>
__global__ void k_objective_seed(Lattice<real> L, const uint8_t* touch, double y_cm, double S, double wcoef, real* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= L.nx) return;
  const int n = y * L.pitch + x;
  double g = 0.0;
  if (L.kind[n] == KIND_FLUID) g = ((double)y - y_cm) / S + (touch[n] ? wcoef : 0.0);
  out[(long long)y * L.nx + x] = (real)g;
}

// lambda = dJ/df of the last state from dJ/drho (row-major nx x ny) and dJ/df (9 such arrays),
// either may be null
template <typename real>
__global__ void k_adj_seed(Lattice<real> L, real* lam, const real* drho, const real* df) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= L.nx) return;
  const int n = y * L.pitch + x;
  const long long c = (long long)y * L.nx + x, dn = (long long)L.nx * L.ny;
  const bool fl = L.kind[n] == KIND_FLUID;
  const real g = fl && drho ? drho[c] : real(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) lam[i * L.plane + n] = fl ? g + (df ? df[i * dn + c] : real(0)) : real(0);
}

// lambda of the first state (nine planes plus the density share), row-major (9 arrays of
// nx x ny; zero off the fluid)
template <typename real>
__global__ void k_adj_export(Lattice<real> L, const real* lam, const real* Lrho, real* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= L.nx) return;
  const int n = y * L.pitch + x;
  const long long c = (long long)y * L.nx + x, dn = (long long)L.nx * L.ny;
  const bool fl = L.kind[n] == KIND_FLUID;
  const real lr = fl ? Lrho[n] : real(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i * dn + c] = fl ? lam[i * L.plane + n] + lr : real(0);
}

// ---- launchers -------------------------------------------------------------------------------
template <typename real>
static dim3 adj_grid(const Lattice<real>& L) { return dim3((unsigned)((L.nx + ADJ_BLOCK - 1) / ADJ_BLOCK), (unsigned)L.ny); }
static unsigned list_grid(int n) { return (unsigned)(n > 0 ? (n + ADJ_BLOCK - 1) / ADJ_BLOCK : 1); }

template <typename real>
cudaError_t adj_flags(const Lattice<real>& L, uint8_t* bct, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bct, 0, (size_t)L.plane, s);
  if (e != cudaSuccess || L.n_bnodes == 0) return e;
  k_adj_flags_x2<real><<<list_grid(L.n_bnodes), ADJ_BLOCK, 0, s>>>(L, bct);
  k_adj_flags_x1<real><<<list_grid(L.n_bnodes), ADJ_BLOCK, 0, s>>>(L, bct);
  return cudaGetLastError();
}

unsigned objective_blocks(long long plane) {
  const long long b = (plane + ADJ_BLOCK - 1) / ADJ_BLOCK;
  return (unsigned)(b < (long long)mass_blocks() ? b : (long long)mass_blocks());
}

template <typename real>
cudaError_t objective_sums(const Lattice<real>& L, int cur, int body, uint8_t* touch, double* red, double rg,
                           double rl, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(touch, 0, (size_t)L.plane, s);
  if (e != cudaSuccess) return e;
  if (L.n_bnodes > 0) k_touch<real><<<list_grid(L.n_bnodes), ADJ_BLOCK, 0, s>>>(L, touch, body);
  k_objective_sums<real><<<objective_blocks(L.plane), ADJ_BLOCK, 0, s>>>(L, cur, touch, red, rg, rl);
  return cudaGetLastError();
}

template <typename real>
cudaError_t objective_seed(const Lattice<real>& L, const uint8_t* touch, double y_cm, double S, double wcoef,
                           real* out, cudaStream_t s) {
  k_objective_seed<real><<<adj_grid(L), ADJ_BLOCK, 0, s>>>(L, touch, y_cm, S, wcoef, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t adj_seed(const Lattice<real>& L, real* lam, const real* drho, const real* df, cudaStream_t s) {
  k_adj_seed<real><<<adj_grid(L), ADJ_BLOCK, 0, s>>>(L, lam, drho, df);
  return cudaGetLastError();
}

template <typename real>
cudaError_t adj_export(const Lattice<real>& L, const real* lam, const real* Lrho, real* out, cudaStream_t s) {
  k_adj_export<real><<<adj_grid(L), ADJ_BLOCK, 0, s>>>(L, lam, Lrho, out);
  return cudaGetLastError();
}

// One reverse step.  L.f[0] holds f^t and L.rho / L.mu the density and chemical potential of
// step t; lambda^{t+1} is (A.lam_in, A.Lrho); leaves lambda^t as (A.lam_out, A.Lrho).
template <typename real>
cudaError_t adj_step(const Lattice<real>& L, const AdjBuffers& A, cudaStream_t s) {
  if (L.n_bnodes > 0) k_adj_bc<real><<<list_grid(L.n_bnodes), ADJ_BLOCK, 0, s>>>(L, A);
  k_adj_collide<real><<<adj_grid(L), ADJ_BLOCK, 0, s>>>(L, A);
  k_adj_force<real><<<adj_grid(L), ADJ_BLOCK, 0, s>>>(L, A);
  k_adj_mu<real><<<adj_grid(L), ADJ_BLOCK, 0, s>>>(L, A);
  if (L.n_s2 > 0) k_adj_solid<real><<<list_grid(L.n_s2), ADJ_BLOCK, 0, s>>>(L, A, 2);
  if (L.n_s1 > 0) k_adj_solid<real><<<list_grid(L.n_s1), ADJ_BLOCK, 0, s>>>(L, A, 1);
  return cudaGetLastError();
}

#define LBMGB_ADJ_INSTANTIATE(real)                                                                        \
  template cudaError_t adj_flags<real>(const Lattice<real>&, uint8_t*, cudaStream_t);                     \
  template cudaError_t objective_sums<real>(const Lattice<real>&, int, int, uint8_t*, double*, double,    \
                                            double, cudaStream_t);                                        \
  template cudaError_t objective_seed<real>(const Lattice<real>&, const uint8_t*, double, double, double, \
                                            real*, cudaStream_t);                                         \
  template cudaError_t adj_seed<real>(const Lattice<real>&, real*, const real*, const real*, cudaStream_t); \
  template cudaError_t adj_export<real>(const Lattice<real>&, const real*, const real*, real*, cudaStream_t); \
  template cudaError_t adj_step<real>(const Lattice<real>&, const AdjBuffers&, cudaStream_t);
LBMGB_ADJ_INSTANTIATE(float)
LBMGB_ADJ_INSTANTIATE(double)

}  // namespace lbmgb
