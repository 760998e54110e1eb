// Host-side equation-of-state set-up of the library (FP64): critical point, pressure,
// bulk chemical potential and Maxwell coexistence densities (Sec. 2.2, Sec. 4 below Eq. 19).
//
// Critical point.  Both EOS are written in a reduced density s (s = eta = b rho/4 for CS,
// s = b rho for PR) as p = RT c1 A(s) - a c2 B(s); the conditions dp/ds = d2p/ds2 = 0 give
// A'(s) B''(s) = A''(s) B'(s), solved for s_c, and RT_c = (a c2 / c1) B'(s_c) / A'(s_c).
//   CS: A = s (1+s+s^2-s^3)/(1-s)^3, c1 = 4/b; B = s^2, c2 = 16/b^2
//   PR: A = s/(1-s), c1 = 1/b; B = s^2/(1+2s-s^2), c2 = 1/b^2   (alpha(Tc) = 1)
// Coexistence.  Newton's method on the saturation pressure p_s for
//   g(p_s) = mu(rho_l(p_s)) - mu(rho_g(p_s)) = 0,  g'(p_s) = 1/rho_l - 1/rho_g
// (Gibbs-Duhem), with rho_g, rho_l the roots of p(rho) = p_s on the gas and liquid branches.
#include <cmath>
#include <cstdio>

#include "lbm_internal.h"

namespace lbmgb {

namespace {

struct Red {
  double A1, A2, B1, B2;  // A', A'', B', B''
};

Red reduced_derivs(int kind, double s) {
  Red r;
  if (kind == EOS_CS) {
    double om = 1.0 - s;
    r.A1 = (1.0 + 4.0 * s + 4.0 * s * s - 4.0 * s * s * s + s * s * s * s) / (om * om * om * om);
    r.A2 = (8.0 + 20.0 * s - 4.0 * s * s) / (om * om * om * om * om);
    r.B1 = 2.0 * s;
    r.B2 = 2.0;
  } else {
    double om = 1.0 - s;
    double D = 1.0 + 2.0 * s - s * s;
    r.A1 = 1.0 / (om * om);
    r.A2 = 2.0 / (om * om * om);
    r.B1 = (2.0 * s + 2.0 * s * s) / (D * D);
    r.B2 = ((2.0 + 4.0 * s) * D - 2.0 * (2.0 * s + 2.0 * s * s) * (2.0 - 2.0 * s)) / (D * D * D);
  }
  return r;
}

double crit_fn(int kind, double s) {
  Red r = reduced_derivs(kind, s);
  return r.A1 * r.B2 - r.A2 * r.B1;
}

// safeguarded Newton for an increasing function on [lo, hi] with f(lo) < 0 < f(hi)
template <class F, class DF>
double newton_bracketed(F f, DF df, double lo, double hi) {
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 300; ++it) {
    double fx = f(x);
    if (fx == 0.0) return x;
    if (fx < 0) lo = x; else hi = x;
    double d = df(x);
    double xn = x - fx / d;
    if (!(xn > lo && xn < hi) || !std::isfinite(xn)) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - x) <= 2e-16 * std::fabs(x) || xn == lo || xn == hi) return xn;
    x = xn;
  }
  return x;
}

}  // namespace

double eos_pressure(int kind, double a, double b, double RT, double aalpha, double rho) {
  if (kind == EOS_CS) {
    double eta = b * rho / 4.0, om = 1.0 - eta;
    return rho * RT * (1.0 + eta + eta * eta - eta * eta * eta) / (om * om * om) - a * rho * rho;
  }
  if (kind == EOS_PR) {
    double x = b * rho;
    return rho * RT / (1.0 - x) - aalpha * rho * rho / (1.0 + 2.0 * x - x * x);
  }
  return rho * RT;
}

static double eos_dpdrho(int kind, double a, double b, double RT, double aalpha, double rho) {
  if (kind == EOS_CS) {
    Red r = reduced_derivs(EOS_CS, b * rho / 4.0);
    return RT * r.A1 - 2.0 * a * rho;
  }
  if (kind == EOS_PR) {
    Red r = reduced_derivs(EOS_PR, b * rho);
    return RT * r.A1 - aalpha / b * r.B1;
  }
  return RT;
}

double eos_mu(int kind, double a, double b, double RT, double aalpha, double rho) {
  if (kind == EOS_CS) {
    double eta = b * rho / 4.0, om = 1.0 - eta;
    return RT * (std::log(rho) + (8.0 * eta - 9.0 * eta * eta + 3.0 * eta * eta * eta) / (om * om * om)) -
           2.0 * a * rho;
  }
  if (kind == EOS_PR) {
    const double s2 = std::sqrt(2.0);
    double x = b * rho;
    return RT * std::log(rho / (1.0 - x)) - aalpha / (2.0 * s2 * b) * std::log((s2 - 1.0 + x) / (s2 + 1.0 - x)) +
           RT / (1.0 - x) - aalpha * rho / (1.0 + 2.0 * x - x * x);
  }
  return RT * std::log(rho);
}

int eos_solve(int kind, double a, double b, double R, double Tr, double omega, EosSolution* out, char* err) {
  EosSolution s{};
  if (kind == EOS_NONE) {
    s.Tc = 1.0; s.T = Tr; s.alpha = 1.0; s.rho_g = s.rho_l = 1.0;
    *out = s;
    return 0;
  }
  if (!(a > 0 && b > 0 && R > 0 && Tr > 0)) {
    std::snprintf(err, 256, "EOS constants a, b, R and T/Tc must be positive");
    return 1;
  }
  // critical point
  double lo = 0.02, hi = kind == EOS_CS ? 0.4 : 0.6;
  double flo = crit_fn(kind, lo), fhi = crit_fn(kind, hi);
  if (flo * fhi > 0) {
    std::snprintf(err, 256, "critical point not bracketed");
    return 1;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    double fm = crit_fn(kind, mid);
    if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
  }
  double sc = 0.5 * (lo + hi);
  Red rc = reduced_derivs(kind, sc);
  double c1 = kind == EOS_CS ? 4.0 / b : 1.0 / b;
  double c2 = kind == EOS_CS ? 16.0 / (b * b) : 1.0 / (b * b);
  double RTc = a * c2 / c1 * rc.B1 / rc.A1;
  s.Tc = RTc / R;
  s.rho_c = kind == EOS_CS ? 4.0 * sc / b : sc / b;
  s.T = Tr * s.Tc;
  const double RT = R * s.T;
  if (kind == EOS_PR) {
    double kw = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
    double q = 1.0 + kw * (1.0 - std::sqrt(Tr));
    s.alpha = q * q;
  } else {
    s.alpha = 1.0;
  }
  const double aal = a * s.alpha;
  auto p = [&](double r) { return eos_pressure(kind, a, b, RT, aal, r); };
  auto dp = [&](double r) { return eos_dpdrho(kind, a, b, RT, aal, r); };
  auto mu = [&](double r) { return eos_mu(kind, a, b, RT, aal, r); };
  const double rmax = kind == EOS_CS ? 4.0 / b : 1.0 / b;
  if (Tr >= 1.0) {
    s.rho_g = s.rho_l = s.rho_c;
    s.mu_sat = mu(s.rho_c);
    s.p_sat = p(s.rho_c);
    *out = s;
    return 0;
  }
  // spinodals: sign changes of dp/drho on a grid, refined by bisection
  const int ng = 20000;
  double s1 = -1, s2 = -1;
  double prev_r = rmax * 1e-9, prev = dp(prev_r);
  for (int k = 1; k <= ng && s2 < 0; ++k) {
    double r = rmax * (0.999 * k / ng);
    double v = dp(r);
    if (s1 < 0 && prev > 0 && v <= 0) {
      double l = prev_r, h = r;
      for (int it = 0; it < 200; ++it) { double m = 0.5 * (l + h); if (m == l || m == h) break; if (dp(m) > 0) l = m; else h = m; }
      s1 = 0.5 * (l + h);
    } else if (s1 > 0 && prev < 0 && v >= 0) {
      double l = prev_r, h = r;
      for (int it = 0; it < 200; ++it) { double m = 0.5 * (l + h); if (m == l || m == h) break; if (dp(m) < 0) l = m; else h = m; }
      s2 = 0.5 * (l + h);
    }
    prev = v;
    prev_r = r;
  }
  if (s1 < 0 || s2 < 0) {
    std::snprintf(err, 256, "no spinodal region: temperature too close to critical");
    return 1;
  }
  auto rho_gas = [&](double ps) {
    return newton_bracketed([&](double r) { return p(r) - ps; }, dp, 1e-300, s1);
  };
  auto rho_liq = [&](double ps) {
    return newton_bracketed([&](double r) { return p(r) - ps; }, dp, s2, rmax * (1.0 - 1e-12));
  };
  double plo = std::fmax(p(s2), p(s1) * 1e-12), phi = p(s1);
  double ps = 0.5 * (plo + phi);
  for (int it = 0; it < 200; ++it) {
    double rg = rho_gas(ps), rl = rho_liq(ps);
    double g = mu(rl) - mu(rg);          // decreasing in ps
    if (g > 0) plo = ps; else phi = ps;
    double dg = 1.0 / rl - 1.0 / rg;
    double pn = ps - g / dg;
    if (!(pn > plo && pn < phi)) pn = 0.5 * (plo + phi);
    if (std::fabs(pn - ps) <= 1e-16 * ps) { ps = pn; break; }
    ps = pn;
  }
  s.p_sat = ps;
  s.rho_g = rho_gas(ps);
  s.rho_l = rho_liq(ps);
  s.mu_sat = mu(s.rho_g);
  *out = s;
  return 0;
}

}  // namespace lbmgb
