// C interface of the reference oracle (TEST INFRASTRUCTURE ONLY; see lbm_oracle.hpp).
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -fPIC -shared
// (-ffp-contract=off: the cut fractions q must be evaluated without fused multiply-adds so
// that they are reproducible bit for bit.)
#include <cstring>
#include <memory>
#include <string>

#include "lbm_oracle.hpp"

using orc::cplx;

extern "C" {

typedef struct {
  int32_t nx, ny;
  int32_t walls;            // 1: solid below y_bottom and above y_top; 0: periodic in y
  double y_bottom, y_top;
  int32_t eos;              // 0 none (body force only), 1 Carnahan-Starling, 2 Peng-Robinson
  double a, b, R, T_over_Tc, omega;
  double k, kappa;          // Eq. 12: mu^ = k^2 psi'(rho) - kappa^ lap(rho)
  int32_t coll;             // 0 BGK, 1 MRT
  double tau, s_e, s_eps, s_q, s_nu;
  double gx, gy;
  int32_t bc;               // 0 present scheme, 1 IBC, 2 MIBC, 3 halfway bounce-back
  int32_t n_cyl;
  const double* cx;
  const double* cy;
  const double* r;
  const double* dmu_w;      // wall chemical potential minus the saturation value (mesh units)
  double dmu_w_walls;
  int32_t force_model;      // 0 chemical potential (Eqs. 9, 12), 1 pseudopotential
} orc_config;

typedef struct {
  int32_t n_drop;
  const double* x0;
  const double* y0;
  const double* r0;
  const double* ux0;
  const double* uy0;
  double width;             // W of Eq. 19
} orc_init_spec;

}  // extern "C"

namespace {

thread_local std::string g_err;

struct Handle {
  int mode = 0;   // 0: double, 1: complex step
  double h = 0;   // complex-step size
  std::unique_ptr<orc::Sim<double>> d;
  std::unique_ptr<orc::Sim<cplx>> c;
};

// adds i*h to v (complex-step instances only)
inline void perturb(double&, double) { throw std::runtime_error("complex step needs a complex instance"); }
inline void perturb(cplx& v, double h) { v += cplx(0.0, h); }

template <class T>
void configure(orc::Sim<T>& s, const orc_config* cfg, int cs_param, int cs_body, double h) {
  if (cfg->nx < 5 || cfg->ny < 5) throw std::runtime_error("grid too small");
  s.nx = cfg->nx;
  s.ny = cfg->ny;
  s.walls = cfg->walls;
  s.yb = cfg->y_bottom;
  s.yt = cfg->y_top;
  if (s.walls) {
    if (!(s.yb >= 1.0 && s.yb < 2.0)) throw std::runtime_error("y_bottom must lie in [1, 2)");
    if (!(s.yt > s.ny - 3.0 && s.yt <= s.ny - 2.0)) throw std::runtime_error("y_top must lie in (ny-3, ny-2]");
  }
  s.eos.kind = cfg->eos;
  s.eos.a = cfg->a;
  s.eos.b = cfg->b;
  s.eos.R = cfg->R;
  s.eos.Tr = cfg->T_over_Tc;
  s.eos.omega = cfg->omega;
  s.eos.k = cfg->k;
  s.eos.kappa = cfg->kappa;
  s.eos.setup();
  s.configure_collision(cfg->coll, cfg->tau, cfg->s_e, cfg->s_eps, cfg->s_q, cfg->s_nu);
  s.gx = cfg->gx;
  s.gy = cfg->gy;
  s.bc = cfg->bc;
  if (cfg->force_model != 0 && cfg->force_model != 1) throw std::runtime_error("force_model must be 0 or 1");
  s.force_model = cfg->force_model;
  s.cx.clear(); s.cy.clear(); s.rad.clear(); s.dmu.clear();
  for (int k = 0; k < cfg->n_cyl; ++k) {
    T cx = cfg->cx[k], cy = cfg->cy[k], dm = cfg->dmu_w[k];
    if (cs_body == k) {
      if (cs_param == 0) perturb(dm, h);
      if (cs_param == 1) perturb(cx, h);
      if (cs_param == 2) perturb(cy, h);
    }
    double r = cfg->r[k];
    if (!(r > 0)) throw std::runtime_error("cylinder radius must be positive");
    if (cfg->cx[k] - r < 2.0 || cfg->cx[k] + r > cfg->nx - 3.0)
      throw std::runtime_error("cylinder must keep two nodes from the periodic x edges");
    if (!cfg->walls && (cfg->cy[k] - r < 2.0 || cfg->cy[k] + r > cfg->ny - 3.0))
      throw std::runtime_error("cylinder must keep two nodes from the periodic y edges");
    s.cx.push_back(cx);
    s.cy.push_back(cy);
    s.rad.push_back(r);
    s.dmu.push_back(dm);
  }
  T dw = cfg->dmu_w_walls;
  if (cs_body == -1 && cs_param == 0) perturb(dw, h);
  s.dmu_walls = dw;
  s.allocate();
  s.build_geometry();
}

Handle* H(void* p) { return static_cast<Handle*>(p); }

template <class F>
int guarded(F&& fn) {
  try {
    fn();
    return 0;
  } catch (const std::exception& e) {
    g_err = e.what();
    return 1;
  }
}

}  // namespace

extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void* orc_create(const orc_config* cfg) {
  Handle* h = new Handle();
  int st = guarded([&] {
    h->mode = 0;
    h->d.reset(new orc::Sim<double>());
    configure<double>(*h->d, cfg, -99, -99, 0.0);
  });
  if (st) { delete h; return nullptr; }
  return h;
}

// Complex-step instance: param 0 perturbs the wall chemical-potential offset of cylinder
// `body` (body -1: the flat walls), 1 its centre x, 2 its centre y, by i*h.
void* orc_create_cs(const orc_config* cfg, int param, int body, double hstep) {
  Handle* h = new Handle();
  int st = guarded([&] {
    h->mode = 1;
    h->h = hstep;
    h->c.reset(new orc::Sim<cplx>());
    configure<cplx>(*h->c, cfg, param, body, hstep);
  });
  if (st) { delete h; return nullptr; }
  return h;
}

void orc_destroy(void* p) { delete H(p); }

int orc_init_droplets(void* p, const orc_init_spec* s) {
  return guarded([&] {
    if (H(p)->mode == 0)
      H(p)->d->init_droplets(s->n_drop, s->x0, s->y0, s->r0, s->ux0, s->uy0, s->width);
    else
      H(p)->c->init_droplets(s->n_drop, s->x0, s->y0, s->r0, s->ux0, s->uy0, s->width);
  });
}

// f = f^eq(rho, u) at fluid nodes from caller arrays of nx*ny doubles
int orc_set_state(void* p, const double* rho, const double* ux, const double* uy) {
  return guarded([&] {
    if (H(p)->mode != 0) throw std::runtime_error("set_state: double instances only");
    auto& s = *H(p)->d;
    std::vector<double> r(rho, rho + s.N()), u(ux, ux + s.N()), v(uy, uy + s.N());
    s.set_state(r, u, v);
  });
}

int orc_step(void* p, int n) {
  return guarded([&] {
    for (int k = 0; k < n; ++k) {
      if (H(p)->mode == 0) H(p)->d->step(); else H(p)->c->step();
    }
  });
}

long long orc_num_links(void* p) {
  return H(p)->mode == 0 ? (long long)H(p)->d->links.size() : (long long)H(p)->c->links.size();
}

int orc_get_links(void* p, int32_t* x1, int32_t* dir, double* q, int32_t* x2, int32_t* x2_fluid) {
  return guarded([&] {
    auto put = [&](auto& s) {
      for (size_t l = 0; l < s.links.size(); ++l) {
        x1[l] = s.links[l].x1;
        dir[l] = s.links[l].dir;
        q[l] = orc::re(s.links[l].q);
        x2[l] = s.links[l].x2;
        x2_fluid[l] = s.links[l].x2_fluid;
      }
    };
    if (H(p)->mode == 0) put(*H(p)->d); else put(*H(p)->c);
  });
}

int orc_get_kind(void* p, uint8_t* kind, int32_t* body) {
  return guarded([&] {
    auto put = [&](auto& s) {
      for (int n = 0; n < s.N(); ++n) { kind[n] = s.kind[n]; body[n] = s.body[n]; }
    };
    if (H(p)->mode == 0) put(*H(p)->d); else put(*H(p)->c);
  });
}

// populations, 9 planes of nx*ny (real parts; imag parts to f_im when given)
int orc_get_f(void* p, double* f, double* f_im) {
  return guarded([&] {
    if (H(p)->mode == 0) {
      auto& s = *H(p)->d;
      std::memcpy(f, s.f.data(), sizeof(double) * s.f.size());
    } else {
      auto& s = *H(p)->c;
      for (size_t k = 0; k < s.f.size(); ++k) {
        f[k] = s.f[k].real();
        if (f_im) f_im[k] = s.f[k].imag();
      }
    }
  });
}

// Overwrite the populations of a double instance (9 planes of nx*ny values, the layout of
// orc_get_f); the step count, the initial mass and the history are kept.  Used by tests that
// perturb the state between steps, e.g. to round it to a storage precision.
int orc_set_f(void* p, const double* f) {
  return guarded([&] {
    if (H(p)->mode != 0) throw std::runtime_error("set_f: double instances only");
    auto& s = *H(p)->d;
    std::memcpy(s.f.data(), f, sizeof(double) * s.f.size());
  });
}

int orc_get_fields(void* p, double* rho, double* vx, double* vy) {
  return guarded([&] {
    if (H(p)->mode == 0) {
      std::vector<double> r, u, v;
      H(p)->d->fields(r, u, v);
      std::memcpy(rho, r.data(), sizeof(double) * r.size());
      std::memcpy(vx, u.data(), sizeof(double) * u.size());
      std::memcpy(vy, v.data(), sizeof(double) * v.size());
    } else {
      std::vector<cplx> r, u, v;
      H(p)->c->fields(r, u, v);
      for (size_t k = 0; k < r.size(); ++k) { rho[k] = r[k].real(); vx[k] = u[k].real(); vy[k] = v[k].real(); }
    }
  });
}

// chemical potential and force of the current state (after orc_get_fields)
int orc_get_mu_force(void* p, double* mu, double* Fx, double* Fy) {
  return guarded([&] {
    if (H(p)->mode != 0) throw std::runtime_error("double instances only");
    auto& s = *H(p)->d;
    std::memcpy(mu, s.mu.data(), sizeof(double) * s.N());
    std::memcpy(Fx, s.Fx.data(), sizeof(double) * s.N());
    std::memcpy(Fy, s.Fy.data(), sizeof(double) * s.N());
  });
}

double orc_mass(void* p) {
  return H(p)->mode == 0 ? H(p)->d->total_mass() : H(p)->c->total_mass().real();
}
double orc_mass0(void* p) {
  return H(p)->mode == 0 ? H(p)->d->mass0 : H(p)->c->mass0.real();
}
long long orc_steps_done(void* p) { return H(p)->mode == 0 ? H(p)->d->steps_done : H(p)->c->steps_done; }

// per-step compensating mass (Eq. 18 summed over the domain) of every step taken so far
int orc_dM_history(void* p, double* out, int n) {
  return guarded([&] {
    const auto& v = H(p)->mode == 0 ? H(p)->d->dM_hist : H(p)->c->dM_hist;
    for (int k = 0; k < n && k < (int)v.size(); ++k) out[k] = v[k];
  });
}

// EOS summary: Tc, rho_c, T, alpha, rho_g, rho_l, mu_sat (= psi'(rho_g)), p_sat
int orc_eos_info(void* p, double* out) {
  return guarded([&] {
    const orc::Eos& e = H(p)->mode == 0 ? H(p)->d->eos : H(p)->c->eos;
    out[0] = e.Tc; out[1] = e.rho_c; out[2] = e.T; out[3] = e.alpha;
    out[4] = e.rho_g; out[5] = e.rho_l; out[6] = e.mu_sat; out[7] = e.p_sat;
  });
}

// EOS evaluation without a simulation: pressure and bulk chemical potential at rho for a
// configuration's EOS (kind, a, b, R, T_over_Tc, omega).
int orc_eos_eval(const orc_config* cfg, int n, const double* rho, double* p, double* mu, double* info8) {
  return guarded([&] {
    orc::Eos e;
    e.kind = cfg->eos; e.a = cfg->a; e.b = cfg->b; e.R = cfg->R; e.Tr = cfg->T_over_Tc;
    e.omega = cfg->omega; e.k = cfg->k; e.kappa = cfg->kappa;
    e.setup();
    for (int j = 0; j < n; ++j) { p[j] = e.pressure(rho[j]); mu[j] = e.psi_prime(rho[j]); }
    if (info8) {
      info8[0] = e.Tc; info8[1] = e.rho_c; info8[2] = e.T; info8[3] = e.alpha;
      info8[4] = e.rho_g; info8[5] = e.rho_l; info8[6] = e.mu_sat; info8[7] = e.p_sat;
    }
  });
}

// droplet objective J = y_cm + L_wet of cylinder `body` for the current state (real and
// imaginary parts; the imaginary part / h is the complex-step derivative)
int orc_objective(void* p, int body, double* J_re, double* J_im) {
  return guarded([&] {
    if (H(p)->mode == 0) {
      auto& s = *H(p)->d;
      if (body < 0 || body >= (int)s.rad.size()) throw std::runtime_error("objective: no such cylinder");
      *J_re = s.objective(body);
      if (J_im) *J_im = 0.0;
    } else {
      auto& s = *H(p)->c;
      if (body < 0 || body >= (int)s.rad.size()) throw std::runtime_error("objective: no such cylinder");
      cplx J = s.objective(body);
      *J_re = J.real();
      if (J_im) *J_im = J.imag();
    }
  });
}

// ---- single-node pieces, for the algebraic pins ----
void orc_mrt_matrices(double* M81, double* Minv81) {
  double inv[9][9];
  orc::invert9(orc::MMAT, inv);
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) { M81[r * 9 + c] = orc::MMAT[r][c]; Minv81[r * 9 + c] = inv[r][c]; }
}

void orc_lattice(int32_t* ex, int32_t* ey, double* w, int32_t* opp) {
  for (int i = 0; i < 9; ++i) { ex[i] = orc::EX[i]; ey[i] = orc::EY[i]; w[i] = orc::WT[i]; opp[i] = orc::opposite(i); }
}

void orc_feq(double rho, double ux, double uy, double* out9) {
  for (int i = 0; i < 9; ++i) out9[i] = orc::feq(i, rho, ux, uy);
}

void orc_meq(double rho, double jx, double jy, double* out9) { orc::meq(rho, jx, jy, out9); }

// one collision (Eq. 4 + Eq. 13) of the populations f9 under force (Fx, Fy)
int orc_collide(const orc_config* cfg, const double* f9, double Fx, double Fy, double* out9, double* Fi9) {
  return guarded([&] {
    orc::Sim<double> s;
    s.nx = 1; s.ny = 1;
    s.configure_collision(cfg->coll, cfg->tau, cfg->s_e, cfg->s_eps, cfg->s_q, cfg->s_nu);
    std::vector<double> fi(9, 0.0);
    double r = 0, jx = 0, jy = 0;
    for (int i = 0; i < 9; ++i) { r += f9[i]; jx += orc::EX[i] * f9[i]; jy += orc::EY[i] * f9[i]; }
    s.collide_node(f9, r, jx / r, jy / r, Fx, Fy, out9, &fi, 0);
    if (Fi9) for (int i = 0; i < 9; ++i) Fi9[i] = fi[i];
  });
}

// Eqs. 16-17 for one link
double orc_link_value(int bc, double q, double a, double b2, int x2_fluid, double c, double F) {
  return orc::Sim<double>::link_value(bc, q, q, a, b2, x2_fluid, c, F);
}

// cut fraction of a cylinder along e_dir from the node (x, y)
double orc_q_cylinder(int x, int y, int dir, double cx, double cy, double r) {
  orc::Sim<double> s;
  s.nx = x + 100000; s.ny = y + 100000; s.walls = 0;
  s.cx.assign(1, cx); s.cy.assign(1, cy); s.rad.assign(1, r); s.dmu.assign(1, 0.0);
  return s.q_body(0, y * s.nx + x, dir);
}

}  // extern "C"
