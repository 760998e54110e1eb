// Device-side building blocks of the multiphase curved-boundary LBM step (sm_103a).
//
// Layout in HBM (one lattice): every per-node quantity is a plane of `pitch * ny` elements,
// node (x, y) at y*pitch + x with pitch = nx rounded up to a 128-byte multiple, so that each
// row starts on a cache-line boundary and a warp touches whole lines.  Populations are 9
// such planes (structure of arrays) per lattice, two lattices A/B swapped every step, stored
// in offset form  f_i - w_i rho_ref.  Padding nodes (x >= nx) carry kind KIND_PAD and are
// never read as data.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lbmgb {

enum : uint8_t { KIND_FLUID = 0, KIND_SOLID1 = 1, KIND_SOLID2 = 2, KIND_DEEP = 3, KIND_PAD = 255 };
enum { EOS_NONE = 0, EOS_CS = 1, EOS_PR = 2 };
enum { COLL_BGK = 0, COLL_MRT = 1 };
enum { BC_PRESENT = 0, BC_IBC = 1, BC_MIBC = 2, BC_HBB = 3 };
constexpr int DM_RING = 4096;

// D2Q9 velocities in the order of the columns of the transformation matrix M (Eq. 2).
__host__ __device__ constexpr int ex(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

// Everything a kernel needs to address one lattice and evaluate its physics.
template <typename real>
struct Lattice {
  int nx, ny, pitch, walls;
  int plane;                    // pitch * ny (9 * plane < 2^31)
  real* f[2];                   // the two population lattices (9 planes each); with aa set both
                                // point at the one lattice, updated in place
  int aa;                       // one lattice (AA order): the state of lattice 0 is in natural
                                // order, that of lattice 1 holds f_i(x) in slot opp(i) of x - e_i
  real* bmom;                   // aa: per boundary node, the pre-collision (delta rho, jx, jy) the
                                // boundary phase needs, saved before the collide overwrites them
  real* rho;                    // density plane (fluid and the two solid layers)
  real* rho_b;                  // if set: the boundary phase leaves the density of each
                                // boundary node's final populations here (one per node)
  real* mu;                     // chemical potential minus k^2 mu_sat (constant at solids)
  real* psip;                   // if set: psi'(rho) - mu_sat of every fluid node, left by the
                                // density pass for the chemical-potential pass (single lattices)
  const uint8_t* kind;
  const int* body;              // body of each solid node (cylinders 0.., then bottom, top wall)
  const double* cyl;            // per cylinder: cx, cy, r, wall chemical-potential offset
  // equation of state, Eq. 12: mu~ = k^2 (psi'(rho) - mu_sat) - kappa lap(rho)
  int eos;
  real RT, a, b, aalpha, k2, kappa, mu_sat;
  real rho_split;                // sqrt(rho_g rho_l): below it mu is evaluated against rho_g
  // CS, per reference density rho0 in {rho_g, rho_l} (index 0 gas, 1 liquid), storage-rounded:
  // rho0, 1/rho0, eta0 = b rho0/4, a0 = 1 - eta0, P(eta0)/a0^3, psi'(rho0) - mu_sat (FP64 on host)
  real cs_r0[2], cs_inv_r0[2], cs_eta0[2], cs_a0[2], cs_p0a3[2], cs_c0[2];
  real rho_ref;
  // collision, Eqs. 3-4
  int coll;
  real omega;                   // 1 / tau (BGK)
  real s_e, s_eps, s_q, s_nu;
  real keep_e, keep_eps, keep_q, keep_nu;   // 1 - s_k, formed once in the storage precision
  real gx, gy;
  int bc;
  // pseudopotential force model (instead of Eqs. 9 and 12): mu holds psi, the solid layers
  // psi(rho_s) (1 + c_w) with c_w = cyl[4 b + 3] of cylinder b, cw_walls of the flat walls
  int pseudo;
  int n_cyl;
  double cw_walls;
  // cut links, CSR over boundary-fluid nodes sorted by node
  int n_bnodes;
  const int* bnode;
  const int* bstart;
  const uint8_t* ldir;
  const real* lq;
  const uint8_t* lx2f;
  // first and second solid layers for Eq. 15
  int n_s1, n_s2;
  const int* s1node;
  const uint8_t* s1mask;         // bit i-1 set: neighbour e_i (i = 1..8) contributes
  const int* s1nb;              // per first-layer entry, 8 ints: the boundary-node index of each
                                // contributing neighbour (-1 elsewhere)
  const real* s1winv;
  const int* s2node;
  const uint8_t* s2mask;
  const real* s2winv;
  double* carry;                // per boundary node: Eq. 18 residual below storage precision
  // reductions (FP64)
  double* partials;             // per-block partial sums
  unsigned int* counter;        // last-block-done counter (returns to 0)
  double* dM_ring;              // per-step domain sum of the Eq. 18 compensation
  unsigned long long* step_ctr; // steps taken (device side)
  double* scalars;              // [0] mass, [1] non-finite count
  unsigned int* kerr;           // set by a kernel whose bounded wait gave up (0 otherwise)
  long long spin_limit;         // polls before a pipelined kernel's wait for its loads gives up
                                // (its wait for copies in flight before leaving keeps the full limit)
  int mu_kernel;                // host side: the chemical-potential pass (0 per node, 1 row
                                // vectors, 2 row sweeps, FP32 only; 3: formed with the next
                                // state's density in one tiled pass, then near_list fixed up)
  int n_near;                   // fluid nodes whose chemical-potential stencil reaches a solid or
  const int* near_list;         // a boundary node (their mu waits for the boundary phase)
  const void* tma;              // host side: TMA descriptors of the pipelined collide kernel
                                // (FP32), null for the plain kernel
  int sweep;                    // host side: the step's collide kernel forms the next state's
                                // density by column sweeps (FP32, chemical-potential force)
  // y-slab of a larger lattice: local row y is global row y + y_off (mod ny_glob when ny_glob >
  // 0); the audits sum rows [own_lo, own_hi) and the Eq. 18 sum boundary nodes [b_lo, b_hi)
  // only.  A whole lattice has y_off = ny_glob = 0, own = [0, ny), b = [0, n_bnodes).
  int y_off, ny_glob;
  int own_lo, own_hi;
  int b_lo, b_hi;
};

// global row of local row y (slabs; the identity for a whole lattice)
template <typename real>
__device__ __forceinline__ int global_row(const Lattice<real>& L, int y) {
  int g = y + L.y_off;
  if (L.ny_glob > 0) g = g < 0 ? g + L.ny_glob : (g >= L.ny_glob ? g - L.ny_glob : g);
  return g;
}

template <typename real>
__device__ __forceinline__ int wrap_x(const Lattice<real>& L, int x) {
  return x < 0 ? x + L.nx : (x >= L.nx ? x - L.nx : x);
}
template <typename real>
__device__ __forceinline__ int wrap_y(const Lattice<real>& L, int y) {
  if (L.walls) return y;
  return y < 0 ? y + L.ny : (y >= L.ny ? y - L.ny : y);
}
template <typename real>
__device__ __forceinline__ int node_at(const Lattice<real>& L, int x, int y) {
  return wrap_y(L, y) * L.pitch + wrap_x(L, x);
}

// Index (into L.f[c]) of population i of node (x, y) of the state held as lattice c: slot i of
// the node, or in AA order (aa, c = 1) slot opp(i) of node (x, y) - e_i.  x, y may lie one node
// outside the lattice (wrapped like node_at).
template <typename real>
__device__ __forceinline__ int pop_index(const Lattice<real>& L, int c, int i, int x, int y) {
  if (L.aa && c == 1) return opp(i) * L.plane + node_at(L, x - ex(i), y - ey(i));
  return i * L.plane + node_at(L, x, y);
}
// the nine populations of node (x, y) of the state held as lattice c
template <typename real>
__device__ __forceinline__ void load_pops(const Lattice<real>& L, int c, int x, int y, real (&fl)[9]) {
  const real* f = L.f[c];
#pragma unroll
  for (int i = 0; i < 9; ++i) fl[i] = f[pop_index(L, c, i, x, y)];
}

// Sums of products with a fixed rounding order.  Where an expression adds two products
// the compiler may fuse either into an FMA, and may choose differently in different kernels;
// the EOS terms, the force and mu are assembled through these, so that every kernel that
// evaluates them (density, scatter, chemical potential, collide, boundary, read-out, batched)
// gets the same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------------------------------
// Equation of state: bulk chemical potential psi'(rho) minus its coexistence value.
//   CS: psi' = RT [ln rho + (8 eta - 9 eta^2 + 3 eta^3)/(1-eta)^3] - 2 a rho,  eta = b rho/4
//   PR: Eq. 11 without the gradient term.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float dev_log(float x) { return logf(x); }
__device__ __forceinline__ double dev_log(double x) { return log(x); }

__device__ __forceinline__ float dev_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double dev_log1p(double x) { return log1p(x); }

// CS: psi'(rho) - mu_sat evaluated against the nearer coexistence density rho0 (gas below
// sqrt(rho_g rho_l), liquid above), where psi'(rho0) = mu_sat:
//   RT ln(rho/rho0) + RT [G(eta) - G(eta0)] - 2a (rho - rho0) + c0,
//   G(eta) = P(eta)/(1-eta)^3,  P = 8 eta - 9 eta^2 + 3 eta^3,
// with ln(rho/rho0) = log1p((rho - rho0)/rho0) and the exact factorisation
//   G(eta) - G(eta0) = h { [8 - 9(eta+eta0) + 3(eta^2 + eta eta0 + eta0^2)] / b^3
//                          + P(eta0) (a^2 + a b + b^2) / (a^3 b^3) },
//   h = eta - eta0, a = 1 - eta0, b = 1 - eta,
// so that every term vanishes with rho - rho0 (which is exact near rho0) instead of cancelling
// between terms of size RT ln rho.  c0 = psi'(rho0) - mu_sat of the storage-rounded rho0 is
// computed in FP64 on the host, so both branches meet the same function.  One division.
template <typename real>
__device__ __forceinline__ real psi_prime_shifted(const Lattice<real>& L, real r) {
  if (L.eos == EOS_CS) {
    const int k = r > L.rho_split ? 1 : 0;
    const real dr = r - L.cs_r0[k];
    const real eta0 = L.cs_eta0[k], a = L.cs_a0[k];
    const real eta = mul_rn(mul_rn(L.b, r), real(0.25));
    const real h = mul_rn(mul_rn(L.b, dr), real(0.25));
    const real bb = real(1) - eta;
    const real ib = real(1) / bb;
    const real ib3 = mul_rn(mul_rn(ib, ib), ib);
    // 8 - 9 (eta + eta0) + 3 (eta^2 + eta eta0 + eta0^2),  P(eta0) (a^2 + a b + b^2) / (a^3 b^3)
    const real sq = fma_rn(eta, eta, fma_rn(eta, eta0, mul_rn(eta0, eta0)));
    const real q1 = fma_rn(real(3), sq, fma_rn(real(-9), eta + eta0, real(8)));
    const real q2 = mul_rn(L.cs_p0a3[k], fma_rn(a, a, fma_rn(a, bb, mul_rn(bb, bb))));
    const real t1 = mul_rn(L.RT, dev_log1p(mul_rn(dr, L.cs_inv_r0[k])));
    const real t2 = mul_rn(mul_rn(L.RT, h), mul_rn(q1 + q2, ib3));
    return (t1 + t2) + fma_rn(mul_rn(real(-2), L.a), dr, L.cs_c0[k]);
  }
  // Peng-Robinson, Eq. 11 without the gradient term
  const real s2 = real(1.4142135623730951);
  const real br = mul_rn(L.b, r);
  const real om = real(1) - br;
  const real t1 = mul_rn(L.RT, dev_log(r / om));
  const real t2 = mul_rn(L.aalpha / mul_rn(real(2) * s2, L.b), dev_log((s2 - real(1) + br) / (s2 + real(1) - br)));
  const real t4 = mul_rn(L.aalpha, r) / fma_rn(-br, br, fma_rn(real(2), br, real(1)));
  return (((t1 - t2) + L.RT / om) - t4) - L.mu_sat;
}

// Fourth-order central first derivatives and Laplacian along the lattice axes.
struct Stencil {
  int xm2, xm1, xp1, xp2, ym2, ym1, yp1, yp2;
};
template <typename real>
__device__ __forceinline__ bool interior(const Lattice<real>& L, int x, int y) {
  // no periodic wrap within two nodes (with walls the rows never wrap: fluid nodes keep two
  // solid rows below and above them)
  return x >= 2 && x < L.nx - 2 && (L.walls || (y >= 2 && y < L.ny - 2));
}

template <typename real>
__device__ __forceinline__ Stencil stencil_at(const Lattice<real>& L, int x, int y) {
  Stencil s;
  if (interior(L, x, y)) {
    const int n = y * L.pitch + x, p = L.pitch;
    s.xm2 = n - 2; s.xm1 = n - 1; s.xp1 = n + 1; s.xp2 = n + 2;
    s.ym2 = n - 2 * p; s.ym1 = n - p; s.yp1 = n + p; s.yp2 = n + 2 * p;
    return s;
  }
  const int row = y * L.pitch;
  s.xm2 = row + wrap_x(L, x - 2);
  s.xm1 = row + wrap_x(L, x - 1);
  s.xp1 = row + wrap_x(L, x + 1);
  s.xp2 = row + wrap_x(L, x + 2);
  s.ym2 = wrap_y(L, y - 2) * L.pitch + x;
  s.ym1 = wrap_y(L, y - 1) * L.pitch + x;
  s.yp1 = wrap_y(L, y + 1) * L.pitch + x;
  s.yp2 = wrap_y(L, y + 2) * L.pitch + x;
  return s;
}

// Undivided fourth-order differences D(p) = 8 (p_1 - p_-1) - (p_2 - p_-2) = 12 dp/dx along
// each axis (8 x exact, so fused or not it rounds the same).
template <typename real>
__device__ __forceinline__ real diff4_of(real p1, real pm1, real p2, real pm2) {
  return real(8) * (p1 - pm1) - (p2 - pm2);
}
template <typename real>
__device__ __forceinline__ void diff4(const real* __restrict__ p, const Stencil& s, real& dx, real& dy) {
  dx = diff4_of(__ldg(p + s.xp1), __ldg(p + s.xm1), __ldg(p + s.xp2), __ldg(p + s.xm2));
  dy = diff4_of(__ldg(p + s.yp1), __ldg(p + s.ym1), __ldg(p + s.yp2), __ldg(p + s.ym2));
}

template <typename real>
__device__ __forceinline__ void grad4(const real* __restrict__ p, const Stencil& s, real& gx, real& gy) {
  const real c = real(1.0 / 12.0);
  gx = (real(8) * (__ldg(p + s.xp1) - __ldg(p + s.xm1)) - (__ldg(p + s.xp2) - __ldg(p + s.xm2))) * c;
  gy = (real(8) * (__ldg(p + s.yp1) - __ldg(p + s.ym1)) - (__ldg(p + s.yp2) - __ldg(p + s.ym2))) * c;
}

// Written as differences from the centre value, (-p2 + 16 p1 - 30 c + 16 p-1 - p-2)/12 =
// (16 [(p1 - c) + (p-1 - c)] - [(p2 - c) + (p-2 - c)])/12: inside a bulk phase the
// differences are exact (Sterbenz), so FP32 keeps the Laplacian's relative accuracy there
// instead of losing it to cancellation between terms of size 30 rho.
template <typename real>
__device__ __forceinline__ real lap4_of(real c, real xp1, real xm1, real xp2, real xm2, real yp1, real ym1, real yp2,
                                        real ym2) {
  real lx = real(16) * ((xp1 - c) + (xm1 - c)) - ((xp2 - c) + (xm2 - c));
  real ly = real(16) * ((yp1 - c) + (ym1 - c)) - ((yp2 - c) + (ym2 - c));
  return (lx + ly) * real(1.0 / 12.0);
}
template <typename real>
__device__ __forceinline__ real lap4(const real* __restrict__ p, int n, const Stencil& s) {
  return lap4_of(p[n], p[s.xp1], p[s.xm1], p[s.xp2], p[s.xm2], p[s.yp1], p[s.ym1], p[s.yp2], p[s.ym2]);
}


// Eq. 12 in mesh units, shifted: mu~ = k^2 (psi'(rho) - mu_sat) - kappa^ lap(rho)
template <typename real>
__device__ __forceinline__ real mu_of(const Lattice<real>& L, real psip, real lap) {
  return fma_rn(L.k2, psip, -mul_rn(L.kappa, lap));
}
// delta rho / 36 to within an ulp: the product with the rounded reciprocal, corrected once
// with its FMA residual
__device__ __forceinline__ float div36(float d) {
  const float c = 1.0f / 36.0f;
  const float q = d * c;
  return fmaf(fmaf(-36.0f, q, d), c, q);
}
__device__ __forceinline__ double div36(double d) { return d / 36.0; }

// F = rho g - rho grad(mu) + c_s^2 grad(rho) (Eq. 9), one component, from the undivided
// differences D(mu) and D(rho) of diff4 (grad = D/12, c_s^2 = 1/3):
//   F = [D(rho) - 3 rho D(mu)] / 36 + rho g.
// Inside an interface the two terms are large and nearly cancel.  The product rho D(mu) enters
// the difference exactly (with its FMA residual), and the division by 36 is corrected to
// within an ulp: no rounded constant (1/12, 1/3) scales either term, because such a constant
// biases the force the same way at every node and step, and that bias builds up in the flow
// where unbiased rounding errors do not.
template <typename real>
__device__ __forceinline__ real force_cp(real r, real g, real dmu, real drho) {
  const real p = mul_rn(r, dmu);
  const real e = fma_rn(r, dmu, -p);
  const real G = fma_rn(real(-3), e, fma_rn(real(-3), p, drho));
  return fma_rn(r, g, div36(G));
}
// F = rho g + c a, the pseudopotential force of centre value c and sum a, one component
template <typename real>
__device__ __forceinline__ real force_pp(real r, real g, real c, real a) {
  return fma_rn(c, a, mul_rn(r, g));
}

// Pseudopotential of the pseudopotential force model, psi = [2 (rho c_s^2 - k^2 p0(rho))]^(1/2)
// clamped at zero (rho c_s^2 + (G/2) psi^2 = k^2 p0 with G = -1), p0 the CS or PR pressure.
template <typename real>
__device__ __forceinline__ real psi_of(const Lattice<real>& L, real r) {
  real p0;
  if (L.eos == EOS_CS) {
    const real eta = mul_rn(mul_rn(L.b, r), real(0.25));
    const real om = real(1) - eta;
    const real poly = fma_rn(eta, fma_rn(eta, real(1) - eta, real(1)), real(1));   // 1 + eta + eta^2 - eta^3
    p0 = mul_rn(mul_rn(r, L.RT), poly) / mul_rn(mul_rn(om, om), om) - mul_rn(mul_rn(L.a, r), r);
  } else {
    const real br = mul_rn(L.b, r);
    p0 = mul_rn(r, L.RT) / (real(1) - br) - mul_rn(mul_rn(L.aalpha, r), r) / fma_rn(br, real(2) - br, real(1));
  }
  const real arg = mul_rn(real(2), fma_rn(r, real(1.0 / 3.0), -mul_rn(L.k2, p0)));
  return arg > real(0) ? sqrt(arg) : real(0);
}

// Adds the pseudopotential force -G psi(x) sum_i w_i psi(x + e_i) e_i (G = -1, w = 1/3 on the
// axes, 1/12 on the diagonals) from the centre value c and the eight neighbours, as
// differences of opposite neighbours (exact inside a bulk phase).
template <typename real>
__device__ __forceinline__ void pp_sums(real e, real n, real w, real s, real ne, real nw, real sw, real se, real& ax,
                                        real& ay) {
  const real d1 = ne - sw, d2 = se - nw;
  const real third = real(1.0 / 3.0), twelfth = real(1.0 / 12.0);
  ax = (e - w) * third + (d1 + d2) * twelfth;
  ay = (n - s) * third + (d1 - d2) * twelfth;
}


// Nonideal force of Eq. 9 in mesh units, F = -rho grad(mu^) + c_s^2 grad(rho), plus rho g;
// with PSEUDO the pseudopotential force from the psi plane instead.
template <typename real, bool PSEUDO = false>
__device__ __forceinline__ void force_at(const Lattice<real>& L, int x, int y, real r, real& Fx, real& Fy) {
  Fx = r * L.gx;
  Fy = r * L.gy;
  if (L.eos == EOS_NONE) return;
  if (PSEUDO) {
    const real* __restrict__ p = L.mu;
    auto at = [&](int dx, int dy) { return __ldg(p + node_at(L, x + dx, y + dy)); };
    real ax, ay;
    pp_sums(at(1, 0), at(0, 1), at(-1, 0), at(0, -1), at(1, 1), at(-1, 1), at(-1, -1), at(1, -1), ax, ay);
    const real c = at(0, 0);
    Fx = force_pp(r, L.gx, c, ax);
    Fy = force_pp(r, L.gy, c, ay);
    return;
  }
  {
    Stencil s = stencil_at(L, x, y);
    real dmx, dmy, drx, dry;
    diff4(L.mu, s, dmx, dmy);
    diff4(L.rho, s, drx, dry);
    Fx = force_cp(r, L.gx, dmx, drx);
    Fy = force_cp(r, L.gy, dmy, dry);
  }
}

// Exact-difference forcing term of Eq. 13 for direction i,
//   F_i = f_i^eq(rho, u + du) - f_i^eq(rho, u),  du = F / rho,
// written as a difference so that FP32 keeps its relative accuracy:
//   w_i rho [3 e.du + 4.5 (e.du)(e.(2u+du)) - 1.5 du.(2u+du)].
template <typename real>
__device__ __forceinline__ real edm_term(int i, real r, real ux, real uy, real dux, real duy) {
  real edu = real(ex(i)) * dux + real(ey(i)) * duy;
  real e2u = real(ex(i)) * (real(2) * ux + dux) + real(ey(i)) * (real(2) * uy + duy);
  real du2u = dux * (real(2) * ux + dux) + duy * (real(2) * uy + duy);
  return real(wgt(i)) * r * (real(3) * edu + real(4.5) * edu * e2u - real(1.5) * du2u);
}

// Moments of a node's offset populations: delta rho = sum_i (f_i - w_i rho_ref) and
// j = sum_i f_i e_i.  j is summed as differences of opposite populations, which are exact in
// floating point near equilibrium (Sterbenz), so the momentum keeps its relative accuracy
// although it is a small difference of populations of size ~rho/9.
template <typename real>
__device__ __forceinline__ real density_sum(const real (&f)[9]) {
  return f[0] + (((f[1] + f[3]) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8])));
}

template <typename real>
__device__ __forceinline__ void moments(const real (&f)[9], real& drho, real& jx, real& jy) {
  drho = density_sum(f);
  jx = (f[1] - f[3]) + ((f[5] - f[7]) + (f[8] - f[6]));
  jy = (f[2] - f[4]) + ((f[5] - f[7]) + (f[6] - f[8]));
}

// Density as the read-out pass and the sweep store it (the same sum, in the same order).
template <typename real>
__device__ __forceinline__ real density_of(const Lattice<real>& L, const real (&f)[9]) {
  return L.rho_ref + density_sum(f);
}

// Collision (Eq. 4) of offset populations with the exact-difference term (Eq. 13).
//   MRT: f~ = f - M^-1 S (m - m_eq) + F_i,  M of Eq. 2, S of Eq. 3, m_eq listed under Eq. 1
//        (q_y^eq = -j_y), all offset by the moments of w_i rho_ref (= m_eq(rho_ref, 0));
//   BGK: f~ = f - (f - f^eq)/tau + F_i.
// The exact-difference term is f^eq(rho, u') - f^eq(rho, u) with u' = u + F/rho, so the
// post-collision populations are f^eq(rho, u') plus the relaxed non-equilibrium part:
//   f~_i = f^eq_i(rho, u') + [M^-1 (I - S) (m - m_eq)]_i,
// M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4); the conserved moments
// drop out.  FP32: the large part of f^eq, w_i delta rho, is formed as {16, 4, 1} x
// (delta rho / 36) -- exact multiples of one quotient, so the weights sum to one exactly and
// no mass bias arises -- and the small terms are added before the final rounding.  The odd
// part of f^eq, w_i rho 3 e_i.u, is formed from the momentum J = rho u itself (odd_split), not
// from rho/9 and rho/36 times u = J/rho: the rounded constants and 1/rho would scale the
// momentum the collision passes on by a fixed factor every step, and at a steady state such a
// bias builds up where unbiased rounding does not.
template <typename real>
__device__ __forceinline__ void odd_split(real Jx, real Jy, real& px, real& py, real& pd, real& pa) {
  // w_i rho 3 e_i.u for e = (1,1) and (-1,1) is (Jx + Jy)/12 and (Jy - Jx)/12; the axis terms
  // take what is left of J/2, so that the first moment of the odd parts is J up to rounding of
  // the sums, whatever the rounding of 1/12
  pd = mul_rn(Jx + Jy, real(1.0 / 12.0));
  pa = mul_rn(Jy - Jx, real(1.0 / 12.0));
  px = fma_rn(real(0.5), Jx, pa - pd);
  py = fma_rn(real(0.5), Jy, -(pd + pa));
}

// The parts added for the odd moments and the BGK branch round every product that meets a sum
// explicitly (mul_rn / fma_rn), so that no kernel's compiler fuses them differently: all kernels
// that collide a node get the same bits.
template <typename real>
__device__ __forceinline__ void collide_node(const Lattice<real>& L, real (&f)[9], real r, real drho,
                                             real jx, real jy, real Fx, real Fy) {
  const real inv_r = real(1) / r;
  const real ux = jx * inv_r, uy = jy * inv_r;
  const real vx = ux + Fx * inv_r, vy = uy + Fy * inv_r;
  const real q36 = div36(drho);
  real neq[9];
  if (L.coll == COLL_MRT) {
    const real s13 = f[1] + f[3], s24 = f[2] + f[4], s57 = f[5] + f[7], s68 = f[6] + f[8];
    const real s1234 = s13 + s24, s5678 = s57 + s68;
    const real d13 = f[1] - f[3], d24 = f[2] - f[4];
    const real j2r = (jx * jx + jy * jy) * inv_r;
    // non-equilibrium moments, scaled by 1 - s_k
    const real e = ((real(-4) * f[0] - s1234 + real(2) * s5678) + (real(2) * drho - real(3) * j2r)) * L.keep_e;
    const real eps = ((real(4) * f[0] - real(2) * s1234 + s5678) - (drho - real(3) * j2r)) * L.keep_eps;
    const real qx = ((jx - real(3) * d13) + jx) * L.keep_q;
    const real qy = ((jy - real(3) * d24) + jy) * L.keep_q;
    const real pxx = ((s13 - s24) - (jx * jx - jy * jy) * inv_r) * L.keep_nu;
    const real pxy = ((s57 - s68) - jx * jy * inv_r) * L.keep_nu;
    const real e36 = e * real(1.0 / 36.0), e18 = e * real(1.0 / 18.0);
    const real s36 = eps * real(1.0 / 36.0), s18 = eps * real(1.0 / 18.0);
    const real qx6 = qx * real(1.0 / 6.0), qy6 = qy * real(1.0 / 6.0);
    const real qx12 = qx * real(1.0 / 12.0), qy12 = qy * real(1.0 / 12.0);
    const real pxx4 = pxx * real(0.25), pxy4 = pxy * real(0.25);
    const real a14 = -e36 - s18, a58 = e18 + s36;
    neq[0] = real(4) * (s36 - e36);
    neq[1] = a14 - qx6 + pxx4;
    neq[2] = a14 - qy6 - pxx4;
    neq[3] = a14 + qx6 + pxx4;
    neq[4] = a14 + qy6 - pxx4;
    neq[5] = a58 + qx12 + qy12 + pxy4;
    neq[6] = a58 - qx12 + qy12 - pxy4;
    neq[7] = a58 - qx12 - qy12 + pxy4;
    neq[8] = a58 + qx12 - qy12 - pxy4;
  } else {
    const real keep = real(1) - L.omega;
    const real usq = mul_rn(real(1.5), fma_rn(ux, ux, mul_rn(uy, uy)));
    real ox, oy, od, oa;
    odd_split(jx, jy, ox, oy, od, oa);
    const real r9 = mul_rn(r, real(1.0 / 9.0)), r36 = mul_rn(r, real(1.0 / 36.0));
    const real ud = ux + uy, ua = uy - ux;
    const real ex_ = fma_rn(mul_rn(real(4.5), ux), ux, -usq), ey_ = fma_rn(mul_rn(real(4.5), uy), uy, -usq);
    const real ed = fma_rn(mul_rn(real(4.5), ud), ud, -usq), ea = fma_rn(mul_rn(real(4.5), ua), ua, -usq);
    neq[0] = mul_rn(keep, (f[0] - real(16) * q36) + real(4) * mul_rn(r9, usq));
    neq[1] = mul_rn(keep, (f[1] - real(4) * q36) - fma_rn(r9, ex_, ox));
    neq[3] = mul_rn(keep, (f[3] - real(4) * q36) - fma_rn(r9, ex_, -ox));
    neq[2] = mul_rn(keep, (f[2] - real(4) * q36) - fma_rn(r9, ey_, oy));
    neq[4] = mul_rn(keep, (f[4] - real(4) * q36) - fma_rn(r9, ey_, -oy));
    neq[5] = mul_rn(keep, (f[5] - q36) - fma_rn(r36, ed, od));
    neq[7] = mul_rn(keep, (f[7] - q36) - fma_rn(r36, ed, -od));
    neq[6] = mul_rn(keep, (f[6] - q36) - fma_rn(r36, ea, oa));
    neq[8] = mul_rn(keep, (f[8] - q36) - fma_rn(r36, ea, -oa));
  }
  // f~_i = w_i delta rho + w_i rho (3 e.u' + 4.5 (e.u')^2 - 1.5 u'^2) + neq_i, opposite
  // directions sharing the even part
  const real vsq = mul_rn(real(1.5), fma_rn(vx, vx, mul_rn(vy, vy)));
  const real r9 = mul_rn(r, real(1.0 / 9.0)), r36 = mul_rn(r, real(1.0 / 36.0));
  // odd parts from the post-collision momentum rho u' = j + F
  real px, py, pd, pa;
  odd_split(jx + Fx, jy + Fy, px, py, pd, pa);
  auto even_of = [&](real ev) { return fma_rn(mul_rn(real(4.5), ev), ev, -vsq); };
  f[0] = real(16) * q36 + (real(-4) * mul_rn(r9, vsq) + neq[0]);
  {
    const real even = even_of(vx);
    f[1] = real(4) * q36 + (fma_rn(r9, even, px) + neq[1]);
    f[3] = real(4) * q36 + (fma_rn(r9, even, -px) + neq[3]);
  }
  {
    const real even = even_of(vy);
    f[2] = real(4) * q36 + (fma_rn(r9, even, py) + neq[2]);
    f[4] = real(4) * q36 + (fma_rn(r9, even, -py) + neq[4]);
  }
  {
    const real even = even_of(vx + vy);
    f[5] = q36 + (fma_rn(r36, even, pd) + neq[5]);
    f[7] = q36 + (fma_rn(r36, even, -pd) + neq[7]);
  }
  {
    const real even = even_of(vy - vx);
    f[6] = q36 + (fma_rn(r36, even, pa) + neq[6]);
    f[8] = q36 + (fma_rn(r36, even, -pa) + neq[8]);
  }
}

// Eqs. 16-17 (present scheme) and their variants for one link.
//   a  = f~_i(x1, t)      (parked in the solid node's slot by the push)
//   b2 = f~_i(x2, t)      (streamed into x1)
//   c  = f~_ibar(x1, t)   (streamed into x2)
//   Fi = F_i(x1, t)       (exact-difference term of direction i at x1)
template <typename real>
__device__ __forceinline__ real link_rule(int bc, real q, int x2_fluid, real a, real b2, real c, real Fi) {
  if (bc == BC_HBB) return a;
  const bool with_force = bc == BC_PRESENT;
  if (q < real(0.5)) {
    if (!x2_fluid) return a;
    real w = real(1) - real(2) * q;
    real v = real(2) * q * a + w * b2;
    if (with_force) v += w * Fi;
    return v;
  }
  real inv = real(1) / (real(2) * q);
  real w = (real(2) * q - real(1)) * inv;
  real v = a * inv + w * c;
  if (with_force) v += w * Fi;
  return v;
}

// Deterministic block sum of one double per thread (fixed shuffle tree, then warps in order).
__device__ __forceinline__ double block_sum(double v, double* smem /* >= 32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double t = 0.0;
  if (warp == 0) {
    t = lane < nw ? smem[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;   // valid in thread 0
}

// Last-block-done finish of a two-level deterministic reduction: every block stores its
// partial; the block that arrives last sums all partials in index order.  Returns true in
// thread 0 of that block, with the total in *total.
__device__ __forceinline__ bool finish_reduction(double block_total, double* partials, unsigned int* counter,
                                                 double* total, double* smem) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = block_total;
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double v = 0.0;
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) v += ((volatile double*)partials)[k];
  double s = block_sum(v, smem);
  if (threadIdx.x == 0) {
    *total = s;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

}  // namespace lbmgb
