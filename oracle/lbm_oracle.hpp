// Reference oracle: a plain, slow, FP64 CPU implementation of one time step of the
// D2Q9 chemical-potential multiphase lattice Boltzmann method with the multiphase curved
// boundary condition of Yao, Liu, Zhong & Wen, "Multiphase curved boundary condition in
// lattice Boltzmann method" (arXiv 2203.04508).
//
// TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA implementation; it shares
// no code, header, table or helper with it.  Only the test-suite, the smoke check and the
// CPU-baseline leg of the benchmark may load it.
//
// Every phase follows the paper's order and notation:
//   Sec. 2.1 (Eqs. 1-5)   MRT / BGK collision and streaming on D2Q9
//   Sec. 2.2 (Eqs. 6-12)  free energy, EOS, chemical potential, nonideal force (Eq. 9),
//                         mesh-space scaling by k (Eq. 12)
//   Sec. 2.2 (Eqs. 13-14) exact-difference forcing
//   Sec. 2.3 (Eq. 15)     chemical-potential wetting boundary (solid-node densities)
//   Sec. 3.1 (Eqs. 16-17) multiphase curved boundary condition, q < 1/2 and q >= 1/2
//   Sec. 3.2 (Eq. 18)     mass compensation of the interpolation error
//   Sec. 4   (Eq. 19)     tanh initial density profile
//
// A second force model replaces Eqs. 9 and 12 by the pseudopotential interaction force that
// the paper cites as the other nonideal-force family (Sec. 1): the Shan-Chen force with the
// pseudopotential built from the EOS (Yuan and Schaefer),
//   F(x) = -G psi(x) sum_i w_i psi(x + e_i) e_i,  G = -1,  w = 1/3 (|e| = 1), 1/12 (|e| = 2^1/2),
//   psi(rho) = sqrt(2 (rho c_s^2 - k^2 p0(rho)) / (-G)),
// so that rho c_s^2 + (G/2) psi^2 is the EOS pressure k^2 p0 in mesh units (the pressure the
// chemical-potential force of Eq. 9 also reproduces).  The exact-difference forcing, the
// collision, the curved boundary (Eqs. 16-18) and Eq. 15 are unchanged; the solid layers carry
// psi(rho_s) (1 + c_w) of their Eq. 15 density rho_s, with the body's wettability parameter c_w
// in place of the wall chemical-potential offset (c_w > -1; positive values make the wall
// hydrophilic, zero is close to neutral).
//
// The scalar type T is double, or std::complex<double> for complex-step derivatives with
// respect to the wall chemical potential and the cylinder centres.  Decisions that are
// discrete (solid or fluid, which branch of Eqs. 16/17) are taken on real parts.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

typedef std::complex<double> cplx;
inline double re(double v) { return v; }
inline double re(const cplx& v) { return v.real(); }

// ---------------------------------------------------------------------------------------
// D2Q9 lattice (Sec. 2.1).  The columns of the transformation matrix M (Eq. 2) fix the
// order of the discrete velocities: rows 4 and 6 of M are the x and y components of e_i.
// The weights are the standard D2Q9 ones that make Eq. 14 the second-order equilibrium with
// c_s^2 = 1/3.
// ---------------------------------------------------------------------------------------
const double MMAT[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},          // rho
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},     // e
    {4, -2, -2, -2, -2, 1, 1, 1, 1},      // epsilon
    {0, 1, 0, -1, 0, 1, -1, -1, 1},       // j_x
    {0, -2, 0, 2, 0, 1, -1, -1, 1},       // q_x
    {0, 0, 1, 0, -1, 1, 1, -1, -1},       // j_y
    {0, 0, -2, 0, 2, 1, 1, -1, -1},       // q_y
    {0, 1, -1, 1, -1, 0, 0, 0, 0},        // p_xx
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};       // p_xy
const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const double WT[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                      1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
const double CS2 = 1.0 / 3.0;

inline int opposite(int i) {
  for (int k = 0; k < 9; ++k)
    if (EX[k] == -EX[i] && EY[k] == -EY[i]) return k;
  return -1;
}

// Inverse of M by Gauss-Jordan elimination with partial pivoting.
inline void invert9(const double A_in[9][9], double inv[9][9]) {
  double a[9][18];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 18; ++c) a[r][c] = c < 9 ? A_in[r][c] : (c - 9 == r ? 1.0 : 0.0);
  for (int c = 0; c < 9; ++c) {
    int piv = c;
    for (int r = c + 1; r < 9; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    for (int k = 0; k < 18; ++k) std::swap(a[c][k], a[piv][k]);
    double d = a[c][c];
    for (int k = 0; k < 18; ++k) a[c][k] /= d;
    for (int r = 0; r < 9; ++r) {
      if (r == c) continue;
      double m = a[r][c];
      if (m == 0.0) continue;
      for (int k = 0; k < 18; ++k) a[r][k] -= m * a[c][k];
    }
  }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) inv[r][c] = a[r][c + 9];
}

// Equilibrium distribution, Eq. 14.
template <class T>
inline T feq(int i, const T& rho, const T& ux, const T& uy) {
  T eu = double(EX[i]) * ux + double(EY[i]) * uy;
  T uu = ux * ux + uy * uy;
  return WT[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

// Equilibria of the moments listed under Eq. 1 (Sec. 2.1).  The printed q_y^(eq) = +j_y is
// read as -j_y: only that sign is consistent with M . f^(eq) of Eq. 14 (q_x^(eq) = -j_x is
// printed with the minus sign, and M treats x and y symmetrically).
template <class T>
inline void meq(const T& rho, const T& jx, const T& jy, T out[9]) {
  T j2 = jx * jx + jy * jy;
  out[0] = rho;
  out[1] = -2.0 * rho + 3.0 * j2 / rho;
  out[2] = rho - 3.0 * j2 / rho;
  out[3] = jx;
  out[4] = -jx;
  out[5] = jy;
  out[6] = -jy;
  out[7] = (jx * jx - jy * jy) / rho;
  out[8] = jx * jy / rho;
}

// ---------------------------------------------------------------------------------------
// Equations of state (Sec. 2.2).
//   kind 0: no nonideal force (ideal gas; the force is the body force only)
//   kind 1: Carnahan-Starling, p0 = rho R T (1+eta+eta^2-eta^3)/(1-eta)^3 - a rho^2,
//           eta = b rho / 4.  Its chemical potential follows from Eq. 7,
//           p0 = rho psi' - psi, i.e. d psi'/d rho = (d p0/d rho) / rho:
//           psi'(rho) = R T [ln rho + (8 eta - 9 eta^2 + 3 eta^3)/(1-eta)^3] - 2 a rho.
//   kind 2: Peng-Robinson, Eq. 10, with chemical potential Eq. 11 (bulk part).
// ---------------------------------------------------------------------------------------
struct Eos {
  int kind = 1;
  double a = 1, b = 4, R = 1, Tr = 0.7, omega = 0.344;
  double k = 1, kappa = 0;
  // derived
  double Tc = 0, rho_c = 0, T = 0, alpha = 1;
  double rho_g = 0, rho_l = 0, mu_sat = 0, p_sat = 0;

  double alpha_of(double Tr_) const {
    if (kind != 2) return 1.0;
    double kw = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
    double s = 1.0 + kw * (1.0 - std::sqrt(Tr_));
    return s * s;
  }
  double rho_max() const { return kind == 1 ? 4.0 / b : 1.0 / b; }

  // Pressure p0 at temperature Tabs with attraction factor alph.
  template <class T2>
  T2 pressure_at(const T2& rho, double Tabs, double alph) const {
    if (kind == 1) {
      T2 eta = b * rho / 4.0;
      T2 om = 1.0 - eta;
      return rho * R * Tabs * (1.0 + eta + eta * eta - eta * eta * eta) / (om * om * om) -
             a * rho * rho;
    }
    if (kind == 2) {
      return rho * R * Tabs / (1.0 - b * rho) -
             a * alph * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
    }
    return rho * R * Tabs;
  }
  // Pseudopotential of the pseudopotential force model: (G/2) psi^2 with G = -1 is the
  // nonideal part k^2 p0 - rho c_s^2 of the mesh pressure.  Where k^2 p0 would exceed
  // rho c_s^2 the radicand is clamped to zero.
  template <class T2>
  T2 pseudopotential(const T2& rho) const {
    T2 arg = 2.0 * (rho / 3.0 - k * k * pressure_at(rho, T, alpha));
    if (re(arg) < 0.0) arg = 0.0;
    using std::sqrt;
    return sqrt(arg);
  }
  // Bulk chemical potential psi'(rho) (the constant of integration is irrelevant: only its
  // gradient enters Eq. 9).
  template <class T2>
  T2 psi_prime_at(const T2& rho, double Tabs, double alph) const {
    using std::log;
    if (kind == 1) {
      T2 eta = b * rho / 4.0;
      T2 om = 1.0 - eta;
      return R * Tabs * (log(rho) + (8.0 * eta - 9.0 * eta * eta + 3.0 * eta * eta * eta) /
                                        (om * om * om)) -
             2.0 * a * rho;
    }
    if (kind == 2) {
      const double s2 = std::sqrt(2.0);
      T2 br = b * rho;
      return R * Tabs * log(rho / (1.0 - br)) -
             a * alph / (2.0 * s2 * b) * log((s2 - 1.0 + br) / (s2 + 1.0 - br)) +
             R * Tabs / (1.0 - br) - a * alph * rho / (1.0 + 2.0 * br - br * br);
    }
    return R * Tabs * log(rho);
  }
  template <class T2>
  T2 psi_prime(const T2& rho) const { return psi_prime_at(rho, T, alpha); }
  double pressure(double rho) const { return pressure_at(rho, T, alpha); }

  // dp0/drho by a complex step (exact to rounding: p0 is analytic in rho).
  double dpdrho_at(double rho, double Tabs, double alph) const {
    const double h = 1e-30;
    cplx z(rho, h);
    return pressure_at(z, Tabs, alph).imag() / h;
  }

  // Minimum of dp0/drho over the physical range: fine scan, then golden section.
  void min_dpdrho(double Tabs, double alph, double* rho_at, double* val) const {
    const int n = 4000;
    double hi = rho_max() * 0.999;
    int best = 1;
    double bv = 1e300;
    for (int k = 1; k < n; ++k) {
      double r = hi * k / n;
      double v = dpdrho_at(r, Tabs, alph);
      if (v < bv) { bv = v; best = k; }
    }
    double lo_r = hi * (best - 1) / n, hi_r = hi * (best + 1) / n;
    const double g = (std::sqrt(5.0) - 1.0) / 2.0;
    double x1 = hi_r - g * (hi_r - lo_r), x2 = lo_r + g * (hi_r - lo_r);
    double f1 = dpdrho_at(x1, Tabs, alph), f2 = dpdrho_at(x2, Tabs, alph);
    for (int it = 0; it < 200; ++it) {
      if (f1 < f2) { hi_r = x2; x2 = x1; f2 = f1; x1 = hi_r - g * (hi_r - lo_r); f1 = dpdrho_at(x1, Tabs, alph); }
      else { lo_r = x1; x1 = x2; f1 = f2; x2 = lo_r + g * (hi_r - lo_r); f2 = dpdrho_at(x2, Tabs, alph); }
    }
    *rho_at = 0.5 * (lo_r + hi_r);
    *val = dpdrho_at(*rho_at, Tabs, alph);
  }

  // Critical point: the temperature at which the minimum of dp0/drho is zero (the
  // attraction factor of Peng-Robinson is alpha(Tc) = 1 there).  Bisection on T.
  void critical_point() {
    if (kind == 0) { Tc = 1.0; rho_c = 0.0; return; }
    double lo = 1e-8, hi = 10.0, r, v;
    for (int it = 0; it < 300; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid == lo || mid == hi) break;
      min_dpdrho(mid, 1.0, &r, &v);
      if (v < 0) lo = mid; else hi = mid;
    }
    Tc = 0.5 * (lo + hi);
    min_dpdrho(Tc, 1.0, &r, &v);
    rho_c = r;
  }

  // Liquid-gas coexistence by the Maxwell equal-area construction (Sec. 4, below Eq. 19):
  // equal pressure and equal chemical potential in the two bulk phases.
  void maxwell() {
    if (kind == 0) { rho_g = rho_l = 1.0; mu_sat = 0.0; p_sat = 0.0; return; }
    double rm, vm;
    min_dpdrho(T, alpha, &rm, &vm);
    if (!(vm < 0)) throw std::runtime_error("temperature is not below the critical point");
    auto dp = [&](double r) { return dpdrho_at(r, T, alpha); };
    auto bisect = [&](auto fn, double lo, double hi) {
      double flo = fn(lo);
      for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        double fm = fn(mid);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
      }
      return 0.5 * (lo + hi);
    };
    // spinodal densities: dp/drho = 0 on each side of the minimum
    double s1 = bisect(dp, 1e-14, rm);
    double s2 = bisect(dp, rm, rho_max() * (1.0 - 1e-12));
    double p_hi = pressure(s1);
    double p_lo = std::max(pressure(s2), p_hi * 1e-12);
    auto rho_gas = [&](double ps) { return bisect([&](double r) { return pressure(r) - ps; }, 1e-300, s1); };
    auto rho_liq = [&](double ps) { return bisect([&](double r) { return pressure(r) - ps; }, s2, rho_max() * (1.0 - 1e-12)); };
    auto gfun = [&](double ps) { return psi_prime(rho_liq(ps)) - psi_prime(rho_gas(ps)); };
    double ps = bisect(gfun, p_lo, p_hi);
    p_sat = ps;
    rho_g = rho_gas(ps);
    rho_l = rho_liq(ps);
    mu_sat = psi_prime(rho_g);
  }

  void setup() {
    critical_point();
    T = Tr * Tc;
    alpha = alpha_of(Tr);
    if (kind != 0 && Tr >= 1.0) {   // supercritical: a single phase
      rho_g = rho_l = rho_c;
      mu_sat = psi_prime(rho_c);
      p_sat = pressure(rho_c);
      return;
    }
    maxwell();
  }
};

// ---------------------------------------------------------------------------------------
// Simulation state and one time step.
// ---------------------------------------------------------------------------------------
enum { BC_PRESENT = 0, BC_IBC = 1, BC_MIBC = 2, BC_HBB = 3 };
enum { KIND_FLUID = 0, KIND_SOLID1 = 1, KIND_SOLID2 = 2, KIND_DEEP = 3 };

template <class T>
struct Link {
  int x1;      // boundary-fluid node (linear index y*nx + x)
  int dir;     // i: direction from x1 towards the solid node x_s = x1 + e_i
  T q;         // fraction of the link x1 -> x_s at which the wall is cut
  int x2;      // x1 - e_i
  int x2_fluid;
};

template <class T>
struct Sim {
  // ---- configuration
  int nx = 0, ny = 0, walls = 0;
  double yb = 0, yt = 0;
  Eos eos;
  int coll = 1;
  double srate[9];
  double tau = 1;
  double gx = 0, gy = 0;
  int bc = BC_PRESENT;
  int force_model = 0;  // 0: chemical potential (Eqs. 9, 12); 1: pseudopotential (see the top)
  std::vector<T> cx, cy;
  std::vector<double> rad;
  std::vector<T> dmu;   // wall chemical potential offsets per cylinder (mesh units)
  T dmu_walls = 0.0;    // the same for the two flat walls
  double Minv[9][9];
  int opp[9];
  // ---- geometry
  std::vector<uint8_t> kind;
  std::vector<int> body;
  std::vector<Link<T>> links;
  std::vector<int> link_start;   // per node: first link index, links are sorted by (x1, dir)
  // ---- state
  std::vector<T> f, ft, fn, Fi;  // 9 planes each, plane i at [i*N, (i+1)*N)
  std::vector<T> rho, mu, ux, uy, Fx, Fy, comp;
  std::vector<double> dM_hist;
  T mass0 = 0.0;
  long steps_done = 0;

  int N() const { return nx * ny; }

  // neighbour of node n along e_i; false if it leaves a non-periodic domain
  bool nb(int n, int i, int* m) const {
    int x = n % nx + EX[i], y = n / nx + EY[i];
    x = (x + nx) % nx;
    if (walls) {
      if (y < 0 || y >= ny) return false;
    } else {
      y = (y + ny) % ny;
    }
    *m = y * nx + x;
    return true;
  }

  int n_bodies() const { return (int)rad.size() + (walls ? 2 : 0); }

  // Is node (x, y) inside body b?  Cylinder: (x-cx)^2 + (y-cy)^2 <= r^2 (boundary nodes
  // count as solid).  Walls: y <= yb (bottom) or y >= yt (top).
  bool inside(int b, int x, int y) const {
    int nc = (int)rad.size();
    if (b < nc) {
      double dx = double(x) - re(cx[b]);
      double dy = double(y) - re(cy[b]);
      double d2 = dx * dx + dy * dy;
      return d2 <= rad[b] * rad[b];
    }
    if (b == nc) return double(y) <= yb;
    return double(y) >= yt;
  }

  // Fraction q of the link from fluid node x1 along e_i at which body b is cut: the smaller
  // root s of |x1 + s e_i - c|^2 = r^2 for a cylinder; the distance to the wall line along
  // the lattice direction for the flat walls.
  T q_body(int b, int n1, int i) const {
    int nc = (int)rad.size();
    int x = n1 % nx, y = n1 / nx;
    if (b < nc) {
      T dx = double(x) - cx[b];
      T dy = double(y) - cy[b];
      double A = double(EX[i] * EX[i] + EY[i] * EY[i]);
      T B = 2.0 * (dx * double(EX[i]) + dy * double(EY[i]));
      T C = (dx * dx + dy * dy) - rad[b] * rad[b];
      T disc = B * B - 4.0 * A * C;
      using std::sqrt;
      return (-B - sqrt(disc)) / (2.0 * A);
    }
    if (b == nc) return T(double(y) - yb);
    return T(yt - double(y));
  }

  void build_geometry() {
    const int n_all = N();
    kind.assign(n_all, KIND_FLUID);
    body.assign(n_all, -1);
    for (int n = 0; n < n_all; ++n) {
      int x = n % nx, y = n / nx;
      for (int b = 0; b < n_bodies(); ++b)
        if (inside(b, x, y)) { body[n] = b; kind[n] = KIND_DEEP; break; }
    }
    // solid layers for Eq. 15 (Sec. 2.3): layer 1 touches a fluid node, layer 2 touches a
    // layer-1 node
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] == KIND_FLUID) continue;
      for (int i = 1; i < 9; ++i) {
        int m;
        if (nb(n, i, &m) && kind[m] == KIND_FLUID) { kind[n] = KIND_SOLID1; break; }
      }
    }
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_DEEP) continue;
      for (int i = 1; i < 9; ++i) {
        int m;
        if (nb(n, i, &m) && kind[m] == KIND_SOLID1) { kind[n] = KIND_SOLID2; break; }
      }
    }
    // every node a fluid stencil (+-1, +-2 along the axes) reaches must exist and carry a
    // density: fluid or one of the two solid layers
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_FLUID) continue;
      int x = n % nx, y = n / nx;
      for (int d = -2; d <= 2; ++d) {
        int yy = y + d;
        if (walls && (yy < 0 || yy >= ny)) throw std::runtime_error("fluid stencil leaves the domain");
        yy = (yy + ny) % ny;
        int xx = ((x + d) % nx + nx) % nx;
        if (kind[yy * nx + x] == KIND_DEEP || kind[y * nx + xx] == KIND_DEEP)
          throw std::runtime_error("fluid stencil reaches a deep solid node");
      }
    }
    // cut links (Sec. 3.1): fluid x1 with x1 + e_i solid, sorted by (x1, i)
    links.clear();
    link_start.assign(n_all + 1, 0);
    for (int n = 0; n < n_all; ++n) {
      link_start[n] = (int)links.size();
      if (kind[n] != KIND_FLUID) continue;
      for (int i = 1; i < 9; ++i) {
        int m;
        if (!nb(n, i, &m)) throw std::runtime_error("fluid node at the domain edge");
        if (kind[m] == KIND_FLUID) continue;
        int xs = m % nx, ys = m / nx;
        bool have = false;
        T qbest = 0.0;
        for (int b = 0; b < n_bodies(); ++b) {
          if (!inside(b, xs, ys)) continue;
          T qb = q_body(b, n, i);
          if (!have || re(qb) < re(qbest)) { qbest = qb; have = true; }
        }
        Link<T> L;
        L.x1 = n;
        L.dir = i;
        L.q = qbest;
        int m2;
        if (!nb(n, opp[i], &m2)) throw std::runtime_error("second interpolation node outside the domain");
        L.x2 = m2;
        L.x2_fluid = kind[m2] == KIND_FLUID ? 1 : 0;
        links.push_back(L);
      }
    }
    link_start[n_all] = (int)links.size();
  }

  void configure_collision(int coll_, double tau_, double se, double seps, double sq, double snu) {
    coll = coll_;
    tau = tau_;
    double s[9] = {1.0, se, seps, 1.0, sq, 1.0, sq, snu, snu};   // Eq. 3
    for (int k = 0; k < 9; ++k) srate[k] = s[k];
    invert9(MMAT, Minv);
    for (int i = 0; i < 9; ++i) opp[i] = opposite(i);
  }

  void allocate() {
    const size_t n = (size_t)N();
    f.assign(9 * n, T(0.0));
    ft.assign(9 * n, T(0.0));
    fn.assign(9 * n, T(0.0));
    Fi.assign(9 * n, T(0.0));
    rho.assign(n, T(0.0));
    mu.assign(n, T(0.0));
    ux.assign(n, T(0.0));
    uy.assign(n, T(0.0));
    Fx.assign(n, T(0.0));
    Fy.assign(n, T(0.0));
    comp.assign(n, T(0.0));
  }

  // Initial state: f = f^(eq)(rho, u) at fluid nodes (Sec. 4).
  void set_state(const std::vector<T>& r, const std::vector<T>& vx, const std::vector<T>& vy) {
    const int n_all = N();
    for (int n = 0; n < n_all; ++n)
      for (int i = 0; i < 9; ++i)
        f[(size_t)i * n_all + n] = kind[n] == KIND_FLUID ? feq(i, r[n], vx[n], vy[n]) : T(0.0);
    mass0 = total_mass();
    steps_done = 0;
    dM_hist.clear();
  }

  // Eq. 19: a tanh profile between the Maxwell densities around each droplet; the droplet
  // with the largest liquid fraction at a node sets its velocity.
  void init_droplets(int nd, const double* x0, const double* y0, const double* r0,
                     const double* u0, const double* v0, double W) {
    const int n_all = N();
    std::vector<T> r(n_all), vx(n_all), vy(n_all);
    for (int n = 0; n < n_all; ++n) {
      double x = n % nx, y = n / nx;
      double phi = 0.0, ux0 = 0.0, uy0 = 0.0;
      for (int d = 0; d < nd; ++d) {
        double dx = x - x0[d], dy = y - y0[d];
        double rr = std::sqrt(dx * dx + dy * dy);
        double ph = 0.5 - 0.5 * std::tanh(2.0 * (rr - r0[d]) / W);
        if (ph > phi) { phi = ph; ux0 = u0 ? u0[d] : 0.0; uy0 = v0 ? v0[d] : 0.0; }
      }
      double dens = 0.5 * (eos.rho_g + eos.rho_l) + 0.5 * (eos.rho_g - eos.rho_l) * (1.0 - 2.0 * phi);
      r[n] = dens;
      vx[n] = ux0 * phi;
      vy[n] = uy0 * phi;
    }
    set_state(r, vx, vy);
  }

  T total_mass() const {
    const int n_all = N();
    T m = 0.0;
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_FLUID) continue;
      for (int i = 0; i < 9; ++i) m += f[(size_t)i * n_all + n];
    }
    return m;
  }

  // ---- phases of one step ----------------------------------------------------------

  // Sec. 2.1: density and momentum, u = j / rho.
  void moments() {
    const int n_all = N();
#pragma omp parallel for schedule(static)
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_FLUID) continue;
      T r = 0.0, jx = 0.0, jy = 0.0;
      for (int i = 0; i < 9; ++i) {
        T fi = f[(size_t)i * n_all + n];
        r += fi;
        jx += double(EX[i]) * fi;
        jy += double(EY[i]) * fi;
      }
      rho[n] = r;
      ux[n] = jx / r;
      uy[n] = jy / r;
    }
  }

  // Eq. 15: density of a solid node as the weighted average of its neighbours of the
  // previous layer (fluid for layer 1, layer 1 for layer 2).
  void solid_density() {
    const int n_all = N();
    for (int layer = KIND_SOLID1; layer <= KIND_SOLID2; ++layer) {
      const int src = layer == KIND_SOLID1 ? KIND_FLUID : KIND_SOLID1;
#pragma omp parallel for schedule(static)
      for (int n = 0; n < n_all; ++n) {
        if (kind[n] != layer) continue;
        T num = 0.0;
        double den = 0.0;
        for (int i = 1; i < 9; ++i) {
          int m;
          if (!nb(n, i, &m) || kind[m] != src) continue;
          num += WT[i] * rho[m];
          den += WT[i];
        }
        rho[n] = num / den;
      }
    }
  }

  // value of a plane at (x + dx, y + dy) of node n
  T at(const std::vector<T>& p, int n, int dx, int dy) const {
    int x = ((n % nx + dx) % nx + nx) % nx;
    int y = n / nx + dy;
    if (!walls) y = ((y % ny) + ny) % ny;
    return p[y * nx + x];
  }
  // fourth-order central first derivatives along the axes
  T ddx(const std::vector<T>& p, int n) const {
    return (8.0 * (at(p, n, 1, 0) - at(p, n, -1, 0)) - (at(p, n, 2, 0) - at(p, n, -2, 0))) / 12.0;
  }
  T ddy(const std::vector<T>& p, int n) const {
    return (8.0 * (at(p, n, 0, 1) - at(p, n, 0, -1)) - (at(p, n, 0, 2) - at(p, n, 0, -2))) / 12.0;
  }
  // fourth-order central Laplacian
  T lap(const std::vector<T>& p, int n) const {
    T c = at(p, n, 0, 0);
    T lx = -at(p, n, 2, 0) + 16.0 * at(p, n, 1, 0) - 30.0 * c + 16.0 * at(p, n, -1, 0) - at(p, n, -2, 0);
    T ly = -at(p, n, 0, 2) + 16.0 * at(p, n, 0, 1) - 30.0 * c + 16.0 * at(p, n, 0, -1) - at(p, n, 0, -2);
    return (lx + ly) / 12.0;
  }

  T wall_mu(int n) const {
    int b = body[n];
    T off = b < (int)rad.size() ? dmu[b] : dmu_walls;
    return eos.k * eos.k * eos.mu_sat + off;
  }

  // Eq. 12 at fluid nodes; the chemical-potential wetting condition at solid nodes.  With
  // the pseudopotential force model this plane holds psi instead: psi(rho) at fluid nodes,
  // psi(rho_s) (1 + c_w) at the solid layers (rho_s from Eq. 15, c_w the body's parameter).
  void chemical_potential() {
    const int n_all = N();
    const double k2 = eos.k * eos.k;
    if (force_model == 1) {
#pragma omp parallel for schedule(static)
      for (int n = 0; n < n_all; ++n) {
        if (kind[n] == KIND_FLUID) {
          mu[n] = eos.pseudopotential(rho[n]);
        } else if (kind[n] == KIND_SOLID1 || kind[n] == KIND_SOLID2) {
          int b = body[n];
          T off = b < (int)rad.size() ? dmu[b] : dmu_walls;
          mu[n] = eos.pseudopotential(rho[n]) * (1.0 + off);
        }
      }
      return;
    }
#pragma omp parallel for schedule(static)
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] == KIND_FLUID)
        mu[n] = k2 * eos.psi_prime(rho[n]) - eos.kappa * lap(rho, n);
      else if (kind[n] == KIND_SOLID1 || kind[n] == KIND_SOLID2)
        mu[n] = wall_mu(n);
    }
  }

  // Eq. 9 plus a body force rho g.
  void force() {
    const int n_all = N();
    const bool nonideal = eos.kind != 0;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_FLUID) continue;
      T fx = rho[n] * gx, fy = rho[n] * gy;
      if (nonideal && force_model == 1) {
        // -G psi(x) sum_i w_i psi(x + e_i) e_i with G = -1; the interaction weights are 3 w_i
        // of the D2Q9 equilibrium (1/3 on the axes, 1/12 on the diagonals)
        T sx = 0.0, sy = 0.0;
        for (int i = 1; i < 9; ++i) {
          T p = at(mu, n, EX[i], EY[i]);
          sx += 3.0 * WT[i] * p * double(EX[i]);
          sy += 3.0 * WT[i] * p * double(EY[i]);
        }
        fx += mu[n] * sx;
        fy += mu[n] * sy;
      } else if (nonideal) {
        fx += -rho[n] * ddx(mu, n) + CS2 * ddx(rho, n);
        fy += -rho[n] * ddy(mu, n) + CS2 * ddy(rho, n);
      }
      Fx[n] = fx;
      Fy[n] = fy;
    }
  }

  // Eq. 4 (MRT: f~ = f - M^-1 S (m - m_eq)) or BGK, plus the exact-difference forcing term
  // of Eq. 13, F_i = f_i^eq(rho, u + F/rho) - f_i^eq(rho, u), with delta t = 1.
  void collide() {
    const int n_all = N();
#pragma omp parallel for schedule(static)
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_FLUID) continue;
      T fl[9], out[9];
      for (int i = 0; i < 9; ++i) fl[i] = f[(size_t)i * n_all + n];
      collide_node(fl, rho[n], ux[n], uy[n], Fx[n], Fy[n], out, &Fi, n);
      for (int i = 0; i < 9; ++i) ft[(size_t)i * n_all + n] = out[i];
    }
  }

  void collide_node(const T fl[9], const T& r, const T& u, const T& v, const T& fx, const T& fy,
                    T out[9], std::vector<T>* fi_store, int n) const {
    const int n_all = N();
    T du = fx / r, dv = fy / r;
    T force_term[9];
    for (int i = 0; i < 9; ++i) force_term[i] = feq(i, r, u + du, v + dv) - feq(i, r, u, v);
    if (coll == 1) {
      T m[9], me[9], ms[9];
      for (int k = 0; k < 9; ++k) {
        m[k] = 0.0;
        for (int i = 0; i < 9; ++i) m[k] += MMAT[k][i] * fl[i];
      }
      meq(r, r * u, r * v, me);
      for (int k = 0; k < 9; ++k) ms[k] = m[k] - srate[k] * (m[k] - me[k]);
      for (int i = 0; i < 9; ++i) {
        T s = 0.0;
        for (int k = 0; k < 9; ++k) s += Minv[i][k] * ms[k];
        out[i] = s + force_term[i];
      }
    } else {
      for (int i = 0; i < 9; ++i) out[i] = fl[i] - (fl[i] - feq(i, r, u, v)) / tau + force_term[i];
    }
    if (fi_store)
      for (int i = 0; i < 9; ++i) (*fi_store)[(size_t)i * n_all + n] = force_term[i];
  }

  // Eq. 5: f_i(x + e_i, t + 1) = f~_i(x, t) between fluid nodes.  Populations that would
  // come from a solid node are left for the boundary condition.
  void stream() {
    const int n_all = N();
#pragma omp parallel for schedule(static)
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_FLUID) continue;
      for (int i = 0; i < 9; ++i) {
        int src;
        T v = 0.0;
        if (nb(n, opp[i], &src) && kind[src] == KIND_FLUID) v = ft[(size_t)i * n_all + src];
        fn[(size_t)i * n_all + n] = v;
      }
    }
  }

  // Eqs. 16-17 for one link.  a = f~_i(x1,t), b2 = f~_i(x2,t), c = f~_ibar(x1,t),
  // F = F_i(x1,t).
  static T link_value(int bc_, double qr, const T& q, const T& a, const T& b2, int x2_fluid,
                      const T& c, const T& F) {
    if (bc_ == BC_HBB) return a;
    const bool with_force = bc_ == BC_PRESENT;
    if (qr < 0.5) {
      if (!x2_fluid) return a;   // no second fluid node to interpolate with: bounce back
      T v = 2.0 * q * a + (1.0 - 2.0 * q) * b2;
      if (with_force) v += (1.0 - 2.0 * q) * F;
      return v;
    }
    T v = a / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * c;
    if (with_force) v += (2.0 * q - 1.0) / (2.0 * q) * F;
    return v;
  }

  // Eqs. 16-18 over the link list.
  void boundary() {
    const int n_all = N();
    const bool compensate = bc == BC_PRESENT || bc == BC_MIBC;
    double dM = 0.0;
    std::vector<T> dm_node(n_all, T(0.0));
#pragma omp parallel for schedule(dynamic, 64)
    for (int n = 0; n < n_all; ++n) {
      T sum = 0.0;
      for (int l = link_start[n]; l < link_start[n + 1]; ++l) {
        const Link<T>& L = links[l];
        const int i = L.dir, ib = opp[i];
        T a = ft[(size_t)i * n_all + L.x1];
        T b2 = L.x2_fluid ? ft[(size_t)i * n_all + L.x2] : T(0.0);
        T c = ft[(size_t)ib * n_all + L.x1];
        T F = Fi[(size_t)i * n_all + L.x1];
        T val = link_value(bc, re(L.q), L.q, a, b2, L.x2_fluid, c, F);
        fn[(size_t)ib * n_all + L.x1] = val;
        sum += a - val;
      }
      if (compensate && link_start[n + 1] > link_start[n]) {
        fn[n] += sum;   // plane 0: the rest population f_0 (Eq. 18)
        dm_node[n] = sum;
      }
    }
    for (int n = 0; n < n_all; ++n) dM += re(dm_node[n]);
    comp.swap(dm_node);
    dM_hist.push_back(dM);
  }

  void step() {
    moments();
    solid_density();
    chemical_potential();
    force();
    collide();
    stream();
    boundary();
    f.swap(fn);
    ++steps_done;
  }

  // Droplet objective of the current state (the gradient target; the paper has none):
  //   J = y_cm + L_wet,
  //   y_cm  = sum_fluid (rho - rho_g) y / sum_fluid (rho - rho_g),  rho = sum_i f_i,
  //   L_wet = (2 pi r_b / N_b) sum over the N_b fluid nodes with a link into body b of
  //           phi(rho) = (rho - rho_g) / (rho_l - rho_g),
  // i.e. the centre-of-mass height of the excess density plus the wetted arc length of the
  // cylinder b estimated from the liquid fraction next to its wall.
  T objective(int b) const {
    const int n_all = N();
    const double rg = eos.rho_g, rl = eos.rho_l;
    T num = 0.0, den = 0.0, wet = 0.0;
    int n_touch = 0;
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_FLUID) continue;
      T r = 0.0;
      for (int i = 0; i < 9; ++i) r += f[(size_t)i * n_all + n];
      num += (r - rg) * double(n / nx);
      den += r - rg;
      bool touches = false;
      for (int l = link_start[n]; l < link_start[n + 1]; ++l) {
        int m;
        nb(n, links[l].dir, &m);
        if (body[m] == b) touches = true;
      }
      if (touches) {
        wet += (r - rg) / (rl - rg);
        ++n_touch;
      }
    }
    const double pi = 3.14159265358979323846;
    T Lw = n_touch > 0 ? (2.0 * pi * rad[b] / double(n_touch)) * wet : T(0.0);
    return num / den + Lw;
  }

  // Macroscopic fields of the current state: rho, and v = u + F/(2 rho) (below Eq. 14).
  void fields(std::vector<T>& r, std::vector<T>& vx, std::vector<T>& vy) {
    moments();
    solid_density();
    chemical_potential();
    force();
    const int n_all = N();
    r.assign(n_all, T(0.0));
    vx.assign(n_all, T(0.0));
    vy.assign(n_all, T(0.0));
    for (int n = 0; n < n_all; ++n) {
      if (kind[n] != KIND_FLUID) continue;
      r[n] = rho[n];
      vx[n] = ux[n] + Fx[n] / (2.0 * rho[n]);
      vy[n] = uy[n] + Fy[n] / (2.0 * rho[n]);
    }
  }
};

}  // namespace orc
