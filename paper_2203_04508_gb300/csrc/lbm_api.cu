// C ABI of the library (declared in include/lbm.h): context, workspace layout, geometry
// set-up, graph-captured time stepping and read-outs.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbmgb;

namespace {

constexpr int MAX_DROPS = 4096;
constexpr int SLAB_MIN_HALO = 7;
constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Caps {
  long long links, bnodes, s1, s2;
};

// Upper bounds of the list sizes.  Nodes of the first / second solid layer and boundary-fluid
// nodes of a cylinder of radius r lie within sqrt(2) resp. 2 sqrt(2) of its circle; the unit
// squares around them are disjoint and lie in the annulus r-3.6 < |x-c| < r+3.2, so its area
// bounds their number.  A node has at most 8 cut links.  Each flat wall has nx nodes per layer
// and 3 cut links per column.
Caps list_caps(const lbm_config* c) {
  Caps k{16, 16, 16, 16};
  for (int j = 0; j < c->n_cyl; ++j) {
    double r = c->r[j];
    double rin = r - 3.6 > 0 ? r - 3.6 : 0.0;
    long long ann = (long long)std::ceil(M_PI * ((r + 3.2) * (r + 3.2) - rin * rin)) + 16;
    k.s1 += ann;
    k.s2 += ann;
    k.bnodes += ann;
    k.links += 8 * ann;
  }
  if (c->walls) {
    k.s1 += 2LL * c->nx;
    k.s2 += 2LL * c->nx;
    k.bnodes += 2LL * c->nx;
    k.links += 6LL * c->nx;
  }
  return k;
}

struct Layout {
  int pitch;
  long long plane;
  size_t sz;
  Caps cap;
  size_t fA, fB, rho, rho2, mu, mu2, psip, kind, body, near, edge, edge_bytes;
  // one lattice (AA order): fB == fA, `stage` holds three planes for the read-outs and the
  // set-up scratch (which use the idle second lattice otherwise), `bmom` the boundary nodes'
  // saved moments
  size_t stage, bmom;
  size_t lq64, lq, ldir, lx2f, bnode, bstart, carry, rhob;
  size_t s1node, s1mask, s1winv, s1nb, s2node, s2mask, s2winv;
  size_t cyl, drops, partials, counter, step_ctr, scalars, kerr, dm_ring, block_sums, totals;
  size_t total;
};

// can the collide kernel form the next density by column sweeps on this lattice?  FP32, the
// chemical-potential force with an equation of state, whole 32 x 8 tiles
bool sweep_shape(const lbm_config* c) {
  return c->precision == LBM_FP32 && c->force_model == LBM_FORCE_CHEMPOT && c->eos != LBM_EOS_NONE && c->nx % 32 == 0 &&
         c->ny % 8 == 0 && c->layout != LBM_LAYOUT_AA;
}

Layout make_layout(const lbm_config* c) {
  Layout L{};
  L.sz = c->precision == LBM_FP64 ? 8 : 4;
  const int per_line = (int)(128 / L.sz);
  L.pitch = (c->nx + per_line - 1) / per_line * per_line;
  L.plane = (long long)L.pitch * c->ny;
  L.cap = list_caps(c);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
  const bool aa = c->layout == LBM_LAYOUT_AA;
  L.fA = take(9 * L.plane * L.sz);
  L.fB = aa ? L.fA : take(9 * L.plane * L.sz);
  L.stage = aa ? take(3 * L.plane * L.sz) : 0;
  L.rho = take(L.plane * L.sz);
  L.rho2 = take(L.plane * L.sz);
  L.mu = take(L.plane * L.sz);
  // the second psi plane (pseudopotential force), or the second mu plane of the FP32 step that
  // forms mu with the next state's density
  L.mu2 = take(c->force_model == LBM_FORCE_PSEUDO || c->precision == LBM_FP32 ? L.plane * L.sz : 0);
  L.psip = take(L.plane * L.sz);
  L.kind = take(L.plane);
  L.body = take(L.plane * 4);
  L.lq64 = take(L.cap.links * 8);
  L.lq = take(L.cap.links * L.sz);
  L.ldir = take(L.cap.links);
  L.lx2f = take(L.cap.links);
  L.bnode = take(L.cap.bnodes * 4);
  L.bstart = take((L.cap.bnodes + 1) * 4);
  L.carry = take(L.cap.bnodes * 8);
  L.rhob = take(L.cap.bnodes * L.sz);
  L.bmom = take(aa ? 3 * L.cap.bnodes * L.sz : 0);
  L.s1node = take(L.cap.s1 * 4);
  L.s1mask = take(L.cap.s1);
  L.s1winv = take(L.cap.s1 * L.sz);
  L.s1nb = take(L.cap.s1 * 8 * 4);
  L.s2node = take(L.cap.s2 * 4);
  L.s2mask = take(L.cap.s2);
  L.s2winv = take(L.cap.s2 * L.sz);
  // fluid nodes whose chemical-potential stencil reaches a solid or boundary node: each solid-layer
  // or boundary node is in the stencils of at most 9 nodes
  L.near = take((size_t)9 * (L.cap.bnodes + L.cap.s1 + L.cap.s2) * 4);
  // edge buffer of the FP32 collide kernel that forms the next density by column sweeps (lattices
  // of whole 32 x 8 tiles, chemical-potential force): nine values per strip-edge node
  L.edge_bytes = sweep_shape(c) ? (size_t)9 * 2 * (c->nx / 32) * c->ny * 4 : 0;
  L.edge = take(L.edge_bytes);
  L.cyl = take((size_t)(c->n_cyl > 0 ? c->n_cyl : 1) * 4 * 8);
  L.drops = take((size_t)MAX_DROPS * 5 * 8);
  size_t nparts = 2 * (size_t)mass_blocks();
  size_t bparts = (size_t)((L.cap.bnodes + 255) / 256) + 1;
  L.partials = take(8 * (nparts > bparts ? nparts : bparts));
  L.counter = take(16);
  L.step_ctr = take(16);
  L.scalars = take(4 * 8);
  L.kerr = take(16);
  L.dm_ring = take((size_t)(DM_RING + 1) * 8);   // the ring, then the last step's value
  L.block_sums = take(((size_t)(L.plane + 1023) / 1024 + 1) * 4 * 5);
  L.totals = take(16 * 4);
  L.total = o;
  return L;
}

}  // namespace

struct lbm_ctx {
  lbm_config cfg{};
  std::vector<double> cx, cy, r, dmu;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  Layout lay{};
  EosSolution eos{};
  bool fp64 = false;
  double rho_ref = 0;
  bool built = false, inited = false;
  int cur = 0;
  // lbm_step keeps the density of lattice `cur` (fluid and solid layers) in density plane `cur`
  // (planes rho, rho2), computing the next one while the boundary phase runs; false until a
  // step or an explicit density pass has put it there
  bool rho_ok = false;
  cudaStream_t side = nullptr;                      // second stream of the overlapped step
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  long long steps = 0;
  long long n_links = 0, n_bnodes = 0, n_s1 = 0, n_s2 = 0, n_fluid = 0;
  Lattice<float> Lf{};
  Lattice<double> Ld{};
  double mass0 = 0;
  // M0 of lbm_init / lbm_set_populations is left on the device (scalars[2]) without waiting for
  // it; the first call that needs it reads it
  bool mass0_pending = false;
  // step graphs (x lattice parity): 2 steps, 1 step, STEPS_LONG steps
  cudaGraphExec_t graph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // FP32: TMA descriptors of the pipelined collide kernel (set up by lbm_build_links) and the
  // collide kernel in use (0 plain, 1 TMA-pipelined, 2 TMA-pipelined column sweeps that form the
  // next density)
  CollideTma tma{};
  bool tma_ok = false;
  int collide_kind = 1;
  long long spin_limit = 1LL << 22;   // polls before a pipelined kernel's wait gives up
  int mu_kind = -1;                   // chemical-potential pass (-1: the precision's default)
  long long n_near = 0;               // entries of the near list, built where the fused density +
  bool near_built = false;            // mu pass is selected (lbm_build_links, lbm_set_mu_kernel)
  lbm_status sticky = LBM_OK;
  std::string err;
  // one segment's recomputation (kind 0) or reverse steps (kind 1), captured once per
  // (workspace, steps, spacing, kind, buffer, length, parity)
  struct AdjGraph {
    const char* ws;
    long long n, every, k;
    int kind, buf, parity;
    cudaGraphExec_t exec;
  };
  std::vector<AdjGraph> adj_graphs;
  // second stream and events of the reverse sweep (created on its first use)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_start = nullptr, ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
  // y-slab of a larger lattice (lbm_create_slab).  Local row y is global row y + y_off (mod
  // the global ny when the global lattice is periodic in y); rows [own_lo, own_hi) are this
  // slab's own; on edge e (0 bottom, 1 top) with a neighbour, rows [recv_lo[e], recv_lo[e] + H)
  // are the halo it receives and [send_lo[e], send_lo[e] + H) the own rows it sends.
  struct Slab {
    bool on = false;
    int y_off = 0, ny_glob = 0, periodic = 0, halo = 0;
    int own_lo = 0, own_hi = 0;
    bool edge[2] = {false, false};
    int recv_lo[2] = {0, 0}, send_lo[2] = {0, 0};
    // boundary-node index ranges of the own rows and of each edge's received and sent rows
    int b_own[2] = {0, 0}, b_recv[2][2] = {{0, 0}, {0, 0}}, b_send[2][2] = {{0, 0}, {0, 0}};
    long long n_fluid_own = 0;
  } slab;
  // the last checkpointed forward pass (lbm_forward_checkpointed), for lbm_adjoint
  struct Tape {
    bool valid = false;
    char* ws = nullptr;
    size_t bytes = 0;
    long long n = 0, every = 0, nseg = 0;
    long long steps_end = 0;
    int cur_end = 0;
  } tape;
};

namespace {

lbm_status fail(lbm_ctx* c, lbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (s == LBM_ECUDA) c->sticky = s;
  }
  return s;
}

#define CUDA_OK(ctx, call)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(ctx, LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));           \
  } while (0)

// The chemical-potential pass by default (FP32): mu formed with the next state's density in one
// tiled pass (kind 3) where both population lattices fit in L2 -- there the step is bound by its
// launches and by the chemical-potential pass's latency, and dropping that pass pays (1024 x 1024:
// 0.0446 against 0.0569 ms a step); on larger lattices the separate passes are faster (2048 x
// 4096: 0.2107 against 0.2255 ms), the row sweeps (kind 2) where their grid of 512-node strips x
// 16-row sweeps fills the GPU four times over, else row vectors (a 512 x 512 lattice gives the
// sweeps only 32 blocks).  FP64: row vectors.
int default_mu_kernel(const lbm_ctx* c) {
  if (c->fp64) return 1;
  int dev = 0, sms = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    sms = 152;
    l2 = 0;
  }
  const bool chempot = c->cfg.force_model == LBM_FORCE_CHEMPOT && c->cfg.eos != LBM_EOS_NONE;
  // (the fused pass reads the populations in 16-byte rows, which the AA order shifts)
  if (chempot && c->cfg.layout != LBM_LAYOUT_AA && 72.0 * c->cfg.nx * c->cfg.ny <= (double)l2) return 3;
  const long long blocks = (long long)((c->cfg.nx + 511) / 512) * ((c->cfg.ny + 15) / 16);
  return blocks >= 4LL * sms ? 2 : 1;
}

template <typename real>
void fill_lattice(lbm_ctx* c, Lattice<real>& L) {
  const Layout& y = c->lay;
  char* w = c->ws;
  L.nx = c->cfg.nx;
  L.ny = c->cfg.ny;
  L.pitch = y.pitch;
  L.walls = c->cfg.walls;
  L.plane = y.plane;
  L.f[0] = (real*)(w + y.fA);
  L.f[1] = (real*)(w + y.fB);
  L.aa = c->cfg.layout == LBM_LAYOUT_AA ? 1 : 0;
  L.bmom = L.aa ? (real*)(w + y.bmom) : nullptr;
  L.rho = (real*)(w + y.rho);
  L.rho_b = nullptr;
  L.mu = (real*)(w + y.mu);
  // the density pass leaves psi'(rho) for the chemical-potential pass (chemical-potential force)
  L.psip = (c->cfg.eos != LBM_EOS_NONE && c->cfg.force_model == LBM_FORCE_CHEMPOT) ? (real*)(w + y.psip) : nullptr;
  L.kind = (const uint8_t*)(w + y.kind);
  L.body = (const int*)(w + y.body);
  L.cyl = (const double*)(w + y.cyl);
  const lbm_config& g = c->cfg;
  L.eos = g.eos;
  const double RT = g.R * c->eos.T;
  L.RT = (real)RT;
  L.a = (real)g.a;
  L.b = (real)g.b;
  L.aalpha = (real)(g.a * c->eos.alpha);
  L.k2 = (real)(g.k * g.k);
  L.kappa = (real)g.kappa;
  L.mu_sat = (real)c->eos.mu_sat;
  L.rho_split = (real)std::sqrt(c->eos.rho_g * c->eos.rho_l);
  for (int k = 0; k < 2; ++k) {
    // reference densities of the CS chemical potential, rounded to the storage type first so
    // that every constant below belongs to the value the kernel actually subtracts
    const real r0 = (real)(k == 0 ? c->eos.rho_g : c->eos.rho_l);
    const double r0d = (double)r0;
    const double eta0 = g.b * r0d / 4.0, a0 = 1.0 - eta0;
    const double P0 = 8.0 * eta0 - 9.0 * eta0 * eta0 + 3.0 * eta0 * eta0 * eta0;
    L.cs_r0[k] = r0;
    L.cs_inv_r0[k] = (real)(1.0 / r0d);
    L.cs_eta0[k] = (real)eta0;
    L.cs_a0[k] = (real)a0;
    L.cs_p0a3[k] = (real)(P0 / (a0 * a0 * a0));
    L.cs_c0[k] = (real)(eos_mu(g.eos, g.a, g.b, RT, g.a * c->eos.alpha, r0d) - c->eos.mu_sat);
  }
  L.rho_ref = (real)c->rho_ref;
  L.coll = g.coll;
  L.omega = (real)(1.0 / g.tau);
  L.s_e = (real)g.s_e;
  L.s_eps = (real)g.s_eps;
  L.s_q = (real)g.s_q;
  L.s_nu = (real)g.s_nu;
  // in the storage precision, as a kernel would form them
  L.keep_e = real(1) - L.s_e;
  L.keep_eps = real(1) - L.s_eps;
  L.keep_q = real(1) - L.s_q;
  L.keep_nu = real(1) - L.s_nu;
  L.gx = (real)g.gx;
  L.gy = (real)g.gy;
  L.bc = g.bc;
  L.pseudo = g.force_model == LBM_FORCE_PSEUDO ? 1 : 0;
  L.n_cyl = g.n_cyl;
  L.cw_walls = g.dmu_w_walls;
  L.n_bnodes = (int)c->n_bnodes;
  L.bnode = (const int*)(w + y.bnode);
  L.bstart = (const int*)(w + y.bstart);
  L.ldir = (const uint8_t*)(w + y.ldir);
  L.lq = (const real*)(w + y.lq);
  L.lx2f = (const uint8_t*)(w + y.lx2f);
  L.carry = (double*)(w + y.carry);
  L.n_s1 = (int)c->n_s1;
  L.n_s2 = (int)c->n_s2;
  L.s1node = (const int*)(w + y.s1node);
  L.s1mask = (const uint8_t*)(w + y.s1mask);
  L.s1winv = (const real*)(w + y.s1winv);
  L.s1nb = (const int*)(w + y.s1nb);
  L.s2node = (const int*)(w + y.s2node);
  L.s2mask = (const uint8_t*)(w + y.s2mask);
  L.s2winv = (const real*)(w + y.s2winv);
  L.partials = (double*)(w + y.partials);
  L.counter = (unsigned int*)(w + y.counter);
  L.dM_ring = (double*)(w + y.dm_ring);
  L.step_ctr = (unsigned long long*)(w + y.step_ctr);
  L.scalars = (double*)(w + y.scalars);
  L.kerr = (unsigned int*)(w + y.kerr);
  L.spin_limit = c->spin_limit;
  L.mu_kernel = c->mu_kind >= 0 ? c->mu_kind : default_mu_kernel(c);
  L.n_near = (int)c->n_near;
  L.near_list = (const int*)(w + y.near);
  L.tma = nullptr;
  if constexpr (sizeof(real) == 4) {
    if (c->tma_ok && c->collide_kind >= 1) L.tma = &c->tma;
  }
  L.sweep = (sizeof(real) == 4 && c->tma_ok && c->collide_kind == 2 && !c->slab.on && sweep_shape(&c->cfg)) ? 1 : 0;
  if (c->slab.on) {
    L.y_off = c->slab.y_off;
    L.ny_glob = c->slab.periodic ? c->slab.ny_glob : 0;
    L.own_lo = c->slab.own_lo;
    L.own_hi = c->slab.own_hi;
    L.b_lo = c->slab.b_own[0];
    L.b_hi = c->slab.b_own[1];
  } else {
    L.y_off = 0;
    L.ny_glob = 0;
    L.own_lo = 0;
    L.own_hi = c->cfg.ny;
    L.b_lo = 0;
    L.b_hi = (int)c->n_bnodes;
  }
}

void refresh(lbm_ctx* c) {
  if (c->fp64) fill_lattice(c, c->Ld); else fill_lattice(c, c->Lf);
}

lbm_status validate(const lbm_config* g, char* msg) {
  auto bad = [&](const char* m) { std::snprintf(msg, 256, "%s", m); return LBM_EINVAL; };
  if (g->nx < 5 || g->ny < 5) return bad("nx and ny must be at least 5");
  if ((long long)g->nx * g->ny > 200000000LL) return bad("lattice larger than 2e8 nodes (32-bit plane offsets)");
  if (g->walls != 0 && g->walls != 1) return bad("walls must be 0 or 1");
  if (g->walls) {
    if (!(g->y_bottom >= 1.0 && g->y_bottom < 2.0)) return bad("y_bottom must lie in [1, 2)");
    if (!(g->y_top > g->ny - 3.0 && g->y_top <= g->ny - 2.0)) return bad("y_top must lie in (ny-3, ny-2]");
  }
  if (g->eos < LBM_EOS_NONE || g->eos > LBM_EOS_PR) return bad("unknown EOS");
  if (g->coll != LBM_COLL_BGK && g->coll != LBM_COLL_MRT) return bad("unknown collision model");
  if (g->bc < LBM_BC_PRESENT || g->bc > LBM_BC_HBB) return bad("unknown boundary scheme");
  if (g->precision != LBM_FP32 && g->precision != LBM_FP64) return bad("precision must be LBM_FP32 or LBM_FP64");
  if (g->coll == LBM_COLL_BGK && !(g->tau > 0.5)) return bad("BGK needs tau > 1/2");
  if (g->coll == LBM_COLL_MRT) {
    const double s[4] = {g->s_e, g->s_eps, g->s_q, g->s_nu};
    for (double v : s)
      if (!(v > 0.0 && v < 2.0)) return bad("MRT rates must lie in (0, 2)");
  }
  if (!(std::isfinite(g->gx) && std::isfinite(g->gy))) return bad("gravity must be finite");
  if (g->eos != LBM_EOS_NONE && !(g->k > 0 && g->kappa >= 0)) return bad("k must be positive and kappa non-negative");
  if (g->n_cyl < 0) return bad("n_cyl must be non-negative");
  if (g->n_cyl > 0 && (!g->cx || !g->cy || !g->r || !g->dmu_w)) return bad("cylinder arrays missing");
  for (int j = 0; j < g->n_cyl; ++j) {
    double r = g->r[j];
    if (!(r > 0)) return bad("cylinder radius must be positive");
    if (g->cx[j] - r < 2.0 || g->cx[j] + r > g->nx - 3.0) return bad("cylinder must keep two nodes from the periodic x edges");
    if (!g->walls && (g->cy[j] - r < 2.0 || g->cy[j] + r > g->ny - 3.0))
      return bad("cylinder must keep two nodes from the periodic y edges");
    if (!std::isfinite(g->dmu_w[j])) return bad("wall chemical potential must be finite");
  }
  if (g->force_model != LBM_FORCE_CHEMPOT && g->force_model != LBM_FORCE_PSEUDO) return bad("unknown force_model");
  if (g->layout != LBM_LAYOUT_AB && g->layout != LBM_LAYOUT_AA) return bad("layout must be LBM_LAYOUT_AB or LBM_LAYOUT_AA");
  if (g->force_model == LBM_FORCE_PSEUDO) {
    // the wall factor c_w multiplies psi by 1 + c_w, which must stay positive
    for (int j = 0; j < g->n_cyl; ++j)
      if (!(g->dmu_w[j] > -1.0)) return bad("pseudopotential wall factor must exceed -1");
    if (!(g->dmu_w_walls > -1.0)) return bad("pseudopotential wall factor must exceed -1");
  }
  return LBM_OK;
}

// descriptors of a step from lattice `cur`: its density in plane `cur`, the boundary densities
// into rho_b, and the next state's density plane
template <typename real>
void step_lattices(const lbm_ctx* c, const Lattice<real>& L, int cur, Lattice<real>& Lt, Lattice<real>& Ln) {
  real* planes[2] = {(real*)(c->ws + c->lay.rho), (real*)(c->ws + c->lay.rho2)};
  Lt = L;
  Lt.rho = planes[cur];
  Lt.rho_b = (real*)(c->ws + c->lay.rhob);
  // psi (pseudopotential force) and mu formed with the density alternate like the density: the
  // next state's is formed while the boundary phase still reads this one's
  const bool alt = c->cfg.force_model == LBM_FORCE_PSEUDO || L.mu_kernel == 3;
  if (alt) {
    real* m[2] = {(real*)(c->ws + c->lay.mu), (real*)(c->ws + c->lay.mu2)};
    Lt.mu = m[cur];
  }
  Ln = Lt;
  Ln.rho = planes[cur ^ 1];
  if (alt) Ln.mu = (real*)(c->ws + (cur ? c->lay.mu : c->lay.mu2));
}

// Steps in the longest step graph (even, so that a launch keeps the lattice parity): fewer
// graph launches, and so fewer gaps between them, for long runs.
constexpr int STEPS_LONG = 8;

// the second stream and events of the overlapped step (created on first use)
lbm_status step_streams(lbm_ctx* c) {
  if (!c->side) {
    CUDA_OK(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  return LBM_OK;
}

// The graph of `steps` (1, 2 or STEPS_LONG) steps from lattice parity p, captured and
// instantiated on first use: slot p (two steps), 2 + p (one) or 4 + p (STEPS_LONG).
template <typename real>
lbm_status step_graph(lbm_ctx* c, const Lattice<real>& L, int p, int steps, cudaGraphExec_t* out) {
  cudaGraphExec_t& slot = c->graph[(steps == 2 ? 0 : steps == 1 ? 2 : 4) + p];
  if (!slot) {
    Lattice<real> Lt, Ln;
    cudaGraph_t g;
    CUDA_OK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaSuccess;
    for (int k = 0; k < steps && e1 == cudaSuccess; ++k) {
      step_lattices(c, L, p ^ (k & 1), Lt, Ln);
      e1 = launch_step_overlap(Lt, Ln, p ^ (k & 1), c->stream, c->side, c->ev_fork, c->ev_join);
    }
    cudaError_t e3 = cudaStreamEndCapture(c->stream, &g);
    if (e1 != cudaSuccess || e3 != cudaSuccess)
      return fail(c, LBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e3));
    cudaError_t e4 = cudaGraphInstantiate(&slot, g, 0);
    cudaGraphDestroy(g);
    if (e4 != cudaSuccess) return fail(c, LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e4));
  }
  *out = slot;
  return LBM_OK;
}

// The graphs lbm_step(n) launches from the current parity, captured without running them.
template <typename real>
lbm_status prepare_steps(lbm_ctx* c, const Lattice<real>& L, long long n) {
  if (n <= 0 || c->stream == nullptr) return LBM_OK;
  lbm_status st = step_streams(c);
  if (st != LBM_OK) return st;
  cudaGraphExec_t g;
  if (n >= STEPS_LONG && (st = step_graph(c, L, c->cur, STEPS_LONG, &g)) != LBM_OK) return st;
  n -= STEPS_LONG * (n / STEPS_LONG);
  if (n >= 2 && (st = step_graph(c, L, c->cur, 2, &g)) != LBM_OK) return st;
  n -= 2 * (n / 2);
  if (n == 1 && (st = step_graph(c, L, c->cur, 1, &g)) != LBM_OK) return st;
  return LBM_OK;
}

template <typename real>
lbm_status do_step(lbm_ctx* c, const Lattice<real>& L, long long n) {
  if (n <= 0) return LBM_OK;
  lbm_status sst = step_streams(c);
  if (sst != LBM_OK) return sst;
  Lattice<real> Lt, Ln;
  if (!c->rho_ok) {
    // density of the current lattice and its solid layers, which the overlapped step expects
    step_lattices(c, L, c->cur, Lt, Ln);
    CUDA_OK(c, launch_phase(Lt, c->cur, 0, c->stream));
    CUDA_OK(c, launch_phase(Lt, c->cur, 1, c->stream));
    // the step that forms mu with the next density starts from this state's mu
    if (L.mu_kernel == 3) CUDA_OK(c, launch_phase(Lt, c->cur, 2, c->stream));
    c->rho_ok = true;
  }
  auto graph_of = [&](int p, int steps, cudaGraphExec_t* out) { return step_graph(c, L, p, steps, out); };
  if (n >= STEPS_LONG && c->stream != nullptr) {
    cudaGraphExec_t gl;
    lbm_status st = graph_of(c->cur, STEPS_LONG, &gl);
    if (st != LBM_OK) return st;
    for (long long k = 0; k < n / STEPS_LONG; ++k) CUDA_OK(c, cudaGraphLaunch(gl, c->stream));
    n -= STEPS_LONG * (n / STEPS_LONG);
  }
  if (n >= 2 && c->stream != nullptr) {
    cudaGraphExec_t g2;
    lbm_status st = graph_of(c->cur, 2, &g2);
    if (st != LBM_OK) return st;
    for (long long k = 0; k < n / 2; ++k) CUDA_OK(c, cudaGraphLaunch(g2, c->stream));
    n -= 2 * (n / 2);
  }
  if (n == 1 && c->stream != nullptr) {
    cudaGraphExec_t g1;
    lbm_status st = graph_of(c->cur, 1, &g1);
    if (st != LBM_OK) return st;
    CUDA_OK(c, cudaGraphLaunch(g1, c->stream));
    c->cur ^= 1;
    n = 0;
  }
  for (long long k = 0; k < n; ++k) {
    step_lattices(c, L, c->cur, Lt, Ln);
    CUDA_OK(c, launch_step_overlap(Lt, Ln, c->cur, c->stream, c->side, c->ev_fork, c->ev_join));
    c->cur ^= 1;
  }
  return LBM_OK;
}

template <typename real>
lbm_status profile_steps(lbm_ctx* c, const Lattice<real>& L, long long n, double* ms) {
  cudaEvent_t ev[6];
  for (auto& e : ev) CUDA_OK(c, cudaEventCreate(&e));
  for (int k = 0; k < 5; ++k) ms[k] = 0.0;
  lbm_status st = LBM_OK;
  if (step_sweeps(L, c->cur)) {
    // the collide kernel forms most of the next density: the phases in the order they depend on
    // one another (chemical potential, collide, boundary links, the next state's solid layers,
    // the densities the collide left), the density planes alternating as lbm_step keeps them
    Lattice<real> Lt, Ln;
    if (!c->rho_ok) {
      step_lattices(c, L, c->cur, Lt, Ln);
      CUDA_OK(c, launch_phase(Lt, c->cur, 0, c->stream));
      CUDA_OK(c, launch_phase(Lt, c->cur, 1, c->stream));
      c->rho_ok = true;
    }
    static const int order[5] = {2, 3, 4, 1, 0};
    for (long long s = 0; s < n && st == LBM_OK; ++s) {
      static const char* const phase_name[5] = {"density", "solid layers", "chemical potential", "collide", "boundary"};
      step_lattices(c, L, c->cur, Lt, Ln);
      for (int k = 0; k < 5; ++k) {
        LBM_RANGE(phase_name[order[k]]);
        cudaEventRecord(ev[k], c->stream);
        cudaError_t e = launch_phase_sweep(Lt, Ln, c->cur, order[k], c->stream);
        if (e != cudaSuccess) { st = fail(c, LBM_ECUDA, "launch failed: %s", cudaGetErrorString(e)); break; }
      }
      if (st != LBM_OK) break;
      cudaEventRecord(ev[5], c->stream);
      cudaError_t e = cudaEventSynchronize(ev[5]);
      if (e != cudaSuccess) { st = fail(c, LBM_ECUDA, "step failed: %s", cudaGetErrorString(e)); break; }
      for (int k = 0; k < 5; ++k) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
        ms[order[k]] += t;
      }
      c->cur ^= 1;
      c->steps += 1;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return st;
  }
  for (long long s = 0; s < n && st == LBM_OK; ++s) {
    static const char* const phase_name[5] = {"density", "solid layers", "chemical potential", "collide", "boundary"};
    for (int ph = 0; ph < 5; ++ph) {
      LBM_RANGE(phase_name[ph]);
      cudaEventRecord(ev[ph], c->stream);
      cudaError_t e = launch_phase(L, c->cur, ph, c->stream);
      if (e != cudaSuccess) { st = fail(c, LBM_ECUDA, "launch failed: %s", cudaGetErrorString(e)); break; }
    }
    cudaEventRecord(ev[5], c->stream);
    cudaError_t e = cudaEventSynchronize(ev[5]);
    if (e != cudaSuccess) { st = fail(c, LBM_ECUDA, "step failed: %s", cudaGetErrorString(e)); break; }
    for (int ph = 0; ph < 5; ++ph) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[ph], ev[ph + 1]);
      ms[ph] += t;
    }
    c->cur ^= 1;
    c->steps += 1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  c->rho_ok = false;   // the phases kept the density in the first plane only
  return st;
}

// Fluid nodes the mass audit counts: a slab's own rows only.
long long fluid_count(const lbm_ctx* c) { return c->slab.on ? c->slab.n_fluid_own : c->n_fluid; }

// The mass audit of the state just set (lbm_init, lbm_set_populations), kept on the device in
// scalars[2..3] (later audits overwrite scalars[0..1]); nothing waits for it.
cudaError_t mass0_async(lbm_ctx* c) {
  cudaError_t e = c->fp64 ? launch_mass(c->Ld, 0, c->stream) : launch_mass(c->Lf, 0, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->ws + c->lay.scalars + 16, c->ws + c->lay.scalars, 16, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) c->mass0_pending = true;
  return e;
}
// M0 on the host, read from the device the first time it is needed (synchronises the stream).
lbm_status resolve_mass0(lbm_ctx* c) {
  if (!c->mass0_pending) return LBM_OK;
  double sc[2];
  CUDA_OK(c, cudaMemcpyAsync(sc, c->ws + c->lay.scalars + 16, 16, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  c->mass0 = sc[0] + (double)fluid_count(c) * c->rho_ref;
  c->mass0_pending = false;
  return LBM_OK;
}

// Device staging memory of the read-outs: the lattice that the next step overwrites completely
// (nine planes), or with one lattice (AA order) the three staging planes.
char* stage_area(const lbm_ctx* c) {
  if (c->cfg.layout == LBM_LAYOUT_AA) return c->ws + c->lay.stage;
  return c->ws + (c->cur ? c->lay.fA : c->lay.fB);
}
// planes of populations the staging memory holds at once
int stage_planes(const lbm_ctx* c) { return c->cfg.layout == LBM_LAYOUT_AA ? 3 : 9; }

// A slab's local configuration: the global one with ny = the rows it holds and flat walls at
// both ends of them -- the global walls where the slab reaches a global wall row, else two
// solid rows beyond the halo at the halfway line (local y 1.5 and ny - 2.5).  Cylinders keep
// their global coordinates; the geometry tests them at global rows.
lbm_status slab_local_config(const lbm_config* g, int y0, int y1, int H, lbm_config* loc, lbm_ctx::Slab* sl,
                             char* msg) {
  auto bad = [&](const char* m) { std::snprintf(msg, 256, "%s", m); return LBM_EINVAL; };
  if (H < SLAB_MIN_HALO) return bad("slab halo must be at least 7 rows (the reach of one step)");
  if (!(0 <= y0 && y0 < y1 && y1 <= g->ny)) return bad("slab rows must satisfy 0 <= y0 < y1 <= ny");
  const int own = y1 - y0;
  const bool bottom = !(g->walls && y0 == 0), top = !(g->walls && y1 == g->ny);
  if ((bottom || top) && own < H) return bad("a slab with a neighbour must own at least halo rows");
  if (g->walls && bottom && y0 < 2) return bad("a walled lattice's wall rows belong to the bottom slab");
  if (g->walls && top && y1 > g->ny - 2) return bad("a walled lattice's wall rows belong to the top slab");
  const int below = bottom ? 2 + H : 0, above = top ? H + 2 : 0;
  *loc = *g;
  loc->ny = own + below + above;
  loc->walls = 1;
  sl->on = true;
  sl->y_off = y0 - below;
  sl->ny_glob = g->ny;
  sl->periodic = g->walls ? 0 : 1;
  sl->halo = H;
  sl->own_lo = below;
  sl->own_hi = below + own;
  sl->edge[0] = bottom;
  sl->edge[1] = top;
  sl->recv_lo[0] = 2;
  sl->send_lo[0] = below;
  sl->recv_lo[1] = below + own;
  sl->send_lo[1] = below + own - H;
  // the global wall lines in local rows (exact: integer shifts of numbers below 2^31)
  loc->y_bottom = bottom ? 1.5 : g->y_bottom - (double)sl->y_off;
  loc->y_top = top ? loc->ny - 2.5 : g->y_top - (double)sl->y_off;
  return LBM_OK;
}

// After the geometry: the boundary-node index ranges of the own rows and of the rows each edge
// sends and receives (the list is sorted by node, so rows are contiguous ranges of it), and the
// fluid nodes of the own rows.
lbm_status slab_ranges(lbm_ctx* c) {
  const Layout& y = c->lay;
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  std::vector<int> bnode(c->n_bnodes > 0 ? c->n_bnodes : 1);
  std::vector<uint8_t> kind(y.plane);
  if (c->n_bnodes > 0)
    CUDA_OK(c, cudaMemcpy(bnode.data(), c->ws + y.bnode, c->n_bnodes * 4, cudaMemcpyDeviceToHost));
  CUDA_OK(c, cudaMemcpy(kind.data(), c->ws + y.kind, y.plane, cudaMemcpyDeviceToHost));
  auto first_at_row = [&](int row) {
    const int key = row * y.pitch;
    return (int)(std::lower_bound(bnode.begin(), bnode.begin() + c->n_bnodes, key) - bnode.begin());
  };
  lbm_ctx::Slab& sl = c->slab;
  sl.b_own[0] = first_at_row(sl.own_lo);
  sl.b_own[1] = first_at_row(sl.own_hi);
  for (int e = 0; e < 2; ++e) {
    sl.b_recv[e][0] = first_at_row(sl.recv_lo[e]);
    sl.b_recv[e][1] = first_at_row(sl.recv_lo[e] + sl.halo);
    sl.b_send[e][0] = first_at_row(sl.send_lo[e]);
    sl.b_send[e][1] = first_at_row(sl.send_lo[e] + sl.halo);
  }
  long long nf = 0;
  for (long long n = (long long)sl.own_lo * y.pitch; n < (long long)sl.own_hi * y.pitch; ++n)
    nf += kind[n] == KIND_FLUID;
  sl.n_fluid_own = nf;
  return LBM_OK;
}

// The fluid nodes whose chemical-potential stencil (the node and two nodes each way along the
// axes) reaches a solid node or a boundary node: the fused density + mu pass cannot finish them,
// since those densities come from the solid-layer kernels and the boundary phase.
lbm_status near_list(lbm_ctx* c) {
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  const Layout& y = c->lay;
  const int nx = c->cfg.nx, ny = c->cfg.ny, P = y.pitch;
  std::vector<uint8_t> kind(y.plane);
  std::vector<int> bnode(c->n_bnodes > 0 ? c->n_bnodes : 1);
  CUDA_OK(c, cudaMemcpy(kind.data(), c->ws + y.kind, y.plane, cudaMemcpyDeviceToHost));
  if (c->n_bnodes > 0) CUDA_OK(c, cudaMemcpy(bnode.data(), c->ws + y.bnode, c->n_bnodes * 4, cudaMemcpyDeviceToHost));
  std::vector<uint8_t> ok(y.plane, 0);   // fluid and not a boundary node
  for (long long n = 0; n < y.plane; ++n) ok[n] = kind[n] == KIND_FLUID;
  for (long long b = 0; b < c->n_bnodes; ++b) ok[bnode[b]] = 0;
  std::vector<int> list;
  for (int yy = 0; yy < ny; ++yy) {
    for (int x = 0; x < nx; ++x) {
      const long long n = (long long)yy * P + x;
      if (kind[n] != KIND_FLUID) continue;
      bool near = !ok[n];
      for (int d = -2; d <= 2 && !near; ++d) {
        if (d == 0) continue;
        const int xx = ((x + d) % nx + nx) % nx;
        int y2 = yy + d;
        if (!c->cfg.walls) y2 = (y2 % ny + ny) % ny;
        near = !ok[(long long)yy * P + xx] || y2 < 0 || y2 >= ny || !ok[(long long)y2 * P + x];
      }
      if (near) list.push_back((int)n);
    }
  }
  const long long cap = 9LL * (y.cap.bnodes + y.cap.s1 + y.cap.s2);
  if ((long long)list.size() > cap)
    return fail(c, LBM_ENOMEM, "near-boundary list of %zu nodes exceeds its capacity %lld", list.size(), cap);
  if (!list.empty())
    CUDA_OK(c, cudaMemcpyAsync(c->ws + y.near, list.data(), list.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
  c->n_near = (long long)list.size();
  c->near_built = true;
  return LBM_OK;
}

// the current density plane and EOS plane (psi'(rho) - mu_sat, or psi) a step starts from
template <typename real>
void slab_planes(const lbm_ctx* c, real** rho, real** aux) {
  *rho = (real*)(c->ws + (c->cur ? c->lay.rho2 : c->lay.rho));
  const int mk = c->fp64 ? c->Ld.mu_kernel : c->Lf.mu_kernel;
  if (c->cfg.force_model == LBM_FORCE_PSEUDO || mk == 3) *aux = (real*)(c->ws + (c->cur ? c->lay.mu2 : c->lay.mu));
  else *aux = (real*)(c->ws + c->lay.psip);
}

lbm_status slab_move(lbm_ctx* c, int32_t edge, void* buf, size_t bytes, bool pack) {
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!c->slab.on) return fail(c, LBM_ESTATE, "not a slab context");
  if (edge != 0 && edge != 1) return fail(c, LBM_EINVAL, "edge must be 0 (bottom) or 1 (top)");
  if (!c->slab.edge[edge]) return fail(c, LBM_EINVAL, "edge %d ends in a wall of the global lattice", edge);
  if (!c->rho_ok) return fail(c, LBM_ESTATE, "exchange halos after a step (the density planes are not current)");
  if (!buf) return fail(c, LBM_EINVAL, "message buffer is NULL");
  const lbm_ctx::Slab& sl = c->slab;
  const size_t need = slab_msg_layout(sl.halo, c->lay.pitch, c->cfg.nx, (int)c->lay.sz).total;
  if (bytes < need) return fail(c, LBM_EINVAL, "message buffer of %zu bytes, %zu needed", bytes, need);
  const int row0 = pack ? sl.send_lo[edge] : sl.recv_lo[edge];
  const int* br = pack ? sl.b_send[edge] : sl.b_recv[edge];
  if (c->fp64) {
    double *rho, *aux;
    slab_planes(c, &rho, &aux);
    CUDA_OK(c, pack ? launch_slab_pack(c->Ld, c->cur, rho, aux, row0, sl.halo, br[0], br[1], buf, c->stream)
                    : launch_slab_unpack(c->Ld, c->cur, rho, aux, row0, sl.halo, br[0], br[1], buf, c->stream));
  } else {
    float *rho, *aux;
    slab_planes(c, &rho, &aux);
    CUDA_OK(c, pack ? launch_slab_pack(c->Lf, c->cur, rho, aux, row0, sl.halo, br[0], br[1], buf, c->stream)
                    : launch_slab_unpack(c->Lf, c->cur, rho, aux, row0, sl.halo, br[0], br[1], buf, c->stream));
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_status_str(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "workspace too small";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ESTATE: return "call out of order";
    case LBM_EUNSTABLE: return "non-finite populations";
    case LBM_ETIMEOUT: return "device wait timed out";
    case LBM_ECORRUPT: return "corrupt checkpoint";
    default: return "internal error";
  }
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }

lbm_status lbm_workspace_size(const lbm_config* cfg, size_t* bytes) {
  if (!cfg || !bytes) return LBM_EINVAL;
  char msg[256];
  lbm_status s = validate(cfg, msg);
  if (s != LBM_OK) return s;
  *bytes = make_layout(cfg).total;
  return LBM_OK;
}

lbm_status lbm_create(const lbm_config* cfg, void* stream, void* workspace, size_t bytes, lbm_ctx** out) {
  LBM_RANGE("lbm_create");
  if (!cfg || !out) return LBM_EINVAL;
  *out = nullptr;
  lbm_ctx* c = new lbm_ctx();
  char msg[256] = {0};
  lbm_status s = validate(cfg, msg);
  if (s != LBM_OK) {
    c->err = msg;
    *out = c;   // returned so that the caller can read lbm_last_error, then destroy
    return s;
  }
  c->cfg = *cfg;
  c->cx.assign(cfg->cx, cfg->cx + cfg->n_cyl);
  c->cy.assign(cfg->cy, cfg->cy + cfg->n_cyl);
  c->r.assign(cfg->r, cfg->r + cfg->n_cyl);
  c->dmu.assign(cfg->dmu_w, cfg->dmu_w + cfg->n_cyl);
  c->cfg.cx = c->cx.data();
  c->cfg.cy = c->cy.data();
  c->cfg.r = c->r.data();
  c->cfg.dmu_w = c->dmu.data();
  c->fp64 = cfg->precision == LBM_FP64;
  if (eos_solve(cfg->eos, cfg->a, cfg->b, cfg->R, cfg->T_over_Tc, cfg->omega, &c->eos, msg)) {
    c->err = msg;
    *out = c;
    return LBM_EINVAL;
  }
  c->rho_ref = cfg->rho_ref >= 0 ? cfg->rho_ref : (c->fp64 ? 0.0 : (cfg->eos == LBM_EOS_NONE ? 1.0 : c->eos.rho_g));
  c->lay = make_layout(&c->cfg);
  *out = c;
  if (!workspace) return fail(c, LBM_EINVAL, "workspace is NULL");
  if (((uintptr_t)workspace) % ALIGN) return fail(c, LBM_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < c->lay.total)
    return fail(c, LBM_ENOMEM, "workspace of %zu bytes, %zu needed", bytes, c->lay.total);
  c->ws = (char*)workspace;
  c->ws_bytes = bytes;
  c->stream = (cudaStream_t)stream;
  refresh(c);
  return LBM_OK;
}

lbm_status lbm_slab_workspace_size(const lbm_config* cfg, int32_t y0, int32_t y1, int32_t halo, size_t* bytes) {
  if (!cfg || !bytes) return LBM_EINVAL;
  char msg[256];
  lbm_status s = validate(cfg, msg);
  if (s != LBM_OK) return s;
  if (cfg->layout != LBM_LAYOUT_AB) return LBM_EINVAL;
  lbm_config loc;
  lbm_ctx::Slab sl;
  s = slab_local_config(cfg, y0, y1, halo, &loc, &sl, msg);
  if (s != LBM_OK) return s;
  *bytes = make_layout(&loc).total;
  return LBM_OK;
}

lbm_status lbm_create_slab(const lbm_config* cfg, int32_t y0, int32_t y1, int32_t halo, void* stream, void* workspace,
                           size_t bytes, lbm_ctx** out) {
  LBM_RANGE("lbm_create_slab");
  if (!cfg || !out) return LBM_EINVAL;
  *out = nullptr;
  char msg[256] = {0};
  lbm_status s = validate(cfg, msg);
  lbm_config loc{};
  lbm_ctx::Slab sl;
  if (s == LBM_OK && cfg->layout != LBM_LAYOUT_AB) {
    std::snprintf(msg, 256, "slabs exchange halos of two population lattices only");
    s = LBM_EINVAL;
  }
  if (s == LBM_OK) s = slab_local_config(cfg, y0, y1, halo, &loc, &sl, msg);
  if (s != LBM_OK) {
    lbm_ctx* c = new lbm_ctx();
    c->err = msg;
    *out = c;
    return s;
  }
  s = lbm_create(&loc, stream, workspace, bytes, out);
  if (*out) {
    (*out)->slab = sl;
    refresh(*out);
  }
  return s;
}

lbm_status lbm_slab_info(lbm_ctx* c, int32_t* info) {
  if (!c || !info) return LBM_EINVAL;
  if (!c->slab.on) return fail(c, LBM_ESTATE, "not a slab context");
  const lbm_ctx::Slab& sl = c->slab;
  const int32_t v[10] = {sl.y_off, c->cfg.ny, sl.own_lo, sl.own_hi, sl.halo, sl.edge[0], sl.edge[1],
                         sl.recv_lo[0], sl.recv_lo[1], sl.periodic};
  std::memcpy(info, v, sizeof(v));
  return LBM_OK;
}

lbm_status lbm_slab_message_bytes(lbm_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LBM_EINVAL;
  if (!c->slab.on) return fail(c, LBM_ESTATE, "not a slab context");
  *bytes = slab_msg_layout(c->slab.halo, c->lay.pitch, c->cfg.nx, (int)c->lay.sz).total;
  return LBM_OK;
}


lbm_status lbm_slab_pack(lbm_ctx* c, int32_t edge, void* buf, size_t bytes) {
  LBM_RANGE("lbm_slab_pack");
  return slab_move(c, edge, buf, bytes, true);
}

lbm_status lbm_slab_unpack(lbm_ctx* c, int32_t edge, const void* buf, size_t bytes) {
  LBM_RANGE("lbm_slab_unpack");
  return slab_move(c, edge, const_cast<void*>(buf), bytes, false);
}

lbm_status lbm_build_links(lbm_ctx* c) {
  LBM_RANGE("lbm_build_links");
  if (!c || !c->ws) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  for (auto& gr : c->graph)
    if (gr) { cudaGraphExecDestroy(gr); gr = nullptr; }
  for (auto& a : c->adj_graphs) cudaGraphExecDestroy(a.exec);
  c->adj_graphs.clear();
  const Layout& y = c->lay;
  const lbm_config& g = c->cfg;
  char* w = c->ws;
  std::vector<double> cyl(4 * (g.n_cyl > 0 ? g.n_cyl : 1), 0.0);
  for (int j = 0; j < g.n_cyl; ++j) {
    cyl[4 * j] = c->cx[j]; cyl[4 * j + 1] = c->cy[j]; cyl[4 * j + 2] = c->r[j]; cyl[4 * j + 3] = c->dmu[j];
  }
  CUDA_OK(c, cudaMemcpyAsync(w + y.cyl, cyl.data(), cyl.size() * 8, cudaMemcpyHostToDevice, c->stream));
  GeomParams gp{};
  gp.nx = g.nx; gp.ny = g.ny; gp.pitch = y.pitch; gp.walls = g.walls; gp.plane = y.plane;
  gp.y_bottom = g.y_bottom; gp.y_top = g.y_top; gp.n_cyl = g.n_cyl; gp.cyl = (const double*)(w + y.cyl);
  gp.dmu_walls = g.dmu_w_walls;
  gp.y_off = c->slab.on ? c->slab.y_off : 0;
  gp.ny_glob = c->slab.on && c->slab.periodic ? c->slab.ny_glob : 0;
  // the second lattice (one lattice: the staging planes) is free until lbm_init: it holds the
  // per-node scratch of the set-up
  GeomScratch sc{};
  sc.body = (int*)(w + y.body);
  sc.cnt = (int*)(w + (c->cfg.layout == LBM_LAYOUT_AA ? y.stage : y.fB));
  sc.off = sc.cnt + y.plane;
  sc.block_sums = (int*)(w + y.block_sums);
  sc.totals = (int*)(w + y.totals);
  CUDA_OK(c, geom_classify_and_count(gp, sc, (uint8_t*)(w + y.kind), c->stream));
  int tot[8];
  CUDA_OK(c, cudaMemcpyAsync(tot, sc.totals, sizeof(tot), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  c->n_links = tot[0]; c->n_bnodes = tot[1]; c->n_s1 = tot[2]; c->n_s2 = tot[3]; c->n_fluid = tot[4];
  if (c->n_links > y.cap.links || c->n_bnodes > y.cap.bnodes || c->n_s1 > y.cap.s1 || c->n_s2 > y.cap.s2)
    return fail(c, LBM_ENOMEM, "geometry exceeds the list capacity (links %lld/%lld)", c->n_links, y.cap.links);
  GeomOut o{};
  o.kind = (uint8_t*)(w + y.kind);
  o.bnode = (int*)(w + y.bnode); o.bstart = (int*)(w + y.bstart); o.ldir = (uint8_t*)(w + y.ldir);
  o.lq64 = (double*)(w + y.lq64); o.lx2f = (uint8_t*)(w + y.lx2f); o.lq = w + y.lq;
  o.s1node = (int*)(w + y.s1node); o.s1mask = (uint8_t*)(w + y.s1mask); o.s1winv = w + y.s1winv;
  o.s1nb = (int*)(w + y.s1nb);
  o.s2node = (int*)(w + y.s2node); o.s2mask = (uint8_t*)(w + y.s2mask); o.s2winv = w + y.s2winv;
  o.mu = w + y.mu;
  o.fp64 = c->fp64;
  o.n_bnodes = (int)c->n_bnodes;
  o.n_s1 = (int)c->n_s1;
  o.n_s2 = (int)c->n_s2;
  CUDA_OK(c, geom_fill(gp, sc, o, 0.0, c->stream));
  int last = (int)c->n_links;
  CUDA_OK(c, cudaMemcpyAsync(o.bstart + c->n_bnodes, &last, 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(c, cudaMemsetAsync(w + y.counter, 0, 16, c->stream));
  CUDA_OK(c, cudaMemsetAsync(w + y.step_ctr, 0, 16, c->stream));
  CUDA_OK(c, cudaMemsetAsync(w + y.kerr, 0, 16, c->stream));
  CUDA_OK(c, cudaMemsetAsync(w + y.dm_ring, 0, (size_t)(DM_RING + 1) * 8, c->stream));
  CUDA_OK(c, cudaMemsetAsync(w + y.rho, 0, y.plane * y.sz, c->stream));
  // the lists are filled on the stream while the host goes on; the calls that read them back
  // (lbm_get_links, lbm_get_kind, the slab ranges, the near-node list) wait for the stream
  if (c->slab.on) {
    lbm_status st = slab_ranges(c);
    if (st != LBM_OK) return st;
  }
  c->n_near = 0;
  c->near_built = false;
  // the second mu plane starts with the walls' constant chemical potential as the first
  if (!c->fp64) CUDA_OK(c, cudaMemcpyAsync(w + y.mu2, w + y.mu, y.plane * y.sz, cudaMemcpyDeviceToDevice, c->stream));
  c->built = true;
  c->inited = false;
  c->rho_ok = false;
  c->tape.valid = false;
  c->tma_ok = false;
  refresh(c);
  if (!c->fp64) {
    // the pipelined collide kernel's descriptors; without them the plain kernel runs
    char msg[256] = {0};
    c->tma_ok = collide_tma_setup(&c->tma, c->Lf, w + y.rho, w + y.rho2, w + y.mu2, y.edge_bytes ? w + y.edge : nullptr,
                                  msg);
    // the pipeline pays off once each persistent block has enough tiles to stream (measured:
    // 43 tiles per block 10 % faster than the plain kernel, 5 tiles per block 7 % slower).  The
    // column sweeps (kind 2) are not the default: on the 2048 x 4096 impact lattice the sweep
    // kernel took 0.24 ms against 0.125 ms (its added density work lands on a kernel already
    // bound by instruction issue) and the step 0.31 ms against 0.21 ms.
    const long long tiles = (long long)((g.nx + 31) / 32) * ((g.ny + 7) / 8);
    c->collide_kind = (c->tma_ok && tiles >= 16LL * c->tma.blocks[g.force_model == LBM_FORCE_PSEUDO ? 1 : 0]) ? 1 : 0;
    refresh(c);
    // the list of nodes the fused density + mu pass leaves to k_mu_near, where that pass runs
    if (c->Lf.mu_kernel == 3) {
      lbm_status st = near_list(c);
      if (st != LBM_OK) return st;
      refresh(c);
    }
  }
  return LBM_OK;
}

lbm_status lbm_counts(lbm_ctx* c, int64_t* nl, int64_t* nb, int64_t* nf, int64_t* n1, int64_t* n2) {
  if (!c || !c->built) return LBM_ESTATE;
  if (nl) *nl = c->n_links;
  if (nb) *nb = c->n_bnodes;
  if (nf) *nf = c->n_fluid;
  if (n1) *n1 = c->n_s1;
  if (n2) *n2 = c->n_s2;
  return LBM_OK;
}

lbm_status lbm_get_links(lbm_ctx* c, int64_t capacity, int32_t* x1, int32_t* dir, double* q, int32_t* x2,
                         int32_t* x2f) {
  if (!c || !c->built) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (capacity < c->n_links) return fail(c, LBM_EINVAL, "capacity %lld < %lld links", (long long)capacity, c->n_links);
  const Layout& y = c->lay;
  const long long L = c->n_links, B = c->n_bnodes;
  std::vector<int> bnode(B), bstart(B + 1);
  std::vector<uint8_t> d(L), f2(L);
  std::vector<double> qq(L);
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  CUDA_OK(c, cudaMemcpy(bnode.data(), c->ws + y.bnode, B * 4, cudaMemcpyDeviceToHost));
  CUDA_OK(c, cudaMemcpy(bstart.data(), c->ws + y.bstart, (B + 1) * 4, cudaMemcpyDeviceToHost));
  CUDA_OK(c, cudaMemcpy(d.data(), c->ws + y.ldir, L, cudaMemcpyDeviceToHost));
  CUDA_OK(c, cudaMemcpy(f2.data(), c->ws + y.lx2f, L, cudaMemcpyDeviceToHost));
  CUDA_OK(c, cudaMemcpy(qq.data(), c->ws + y.lq64, L * 8, cudaMemcpyDeviceToHost));
  const int nx = c->cfg.nx, ny = c->cfg.ny;
  for (long long b = 0; b < B; ++b) {
    int n = bnode[b];
    int x = n % y.pitch, yy = n / y.pitch;
    for (int l = bstart[b]; l < bstart[b + 1]; ++l) {
      int i = d[l];
      if (x1) x1[l] = yy * nx + x;
      if (dir) dir[l] = i;
      if (q) q[l] = qq[l];
      int xx = ((x - ex(i)) % nx + nx) % nx;
      int y2 = yy - ey(i);
      if (!c->cfg.walls) y2 = (y2 % ny + ny) % ny;
      if (x2) x2[l] = y2 * nx + xx;
      if (x2f) x2f[l] = f2[l];
    }
  }
  return LBM_OK;
}

lbm_status lbm_get_kind(lbm_ctx* c, uint8_t* kind) {
  if (!c || !c->built) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  const Layout& y = c->lay;
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  CUDA_OK(c, cudaMemcpy2D(kind, c->cfg.nx, c->ws + y.kind, y.pitch, c->cfg.nx, c->cfg.ny, cudaMemcpyDeviceToHost));
  return LBM_OK;
}

lbm_status lbm_init(lbm_ctx* c, const lbm_init_spec* s) {
  LBM_RANGE("lbm_init");
  if (!c || !c->built) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!s || s->n_drop < 0 || s->n_drop > MAX_DROPS) return fail(c, LBM_EINVAL, "n_drop must lie in [0, %d]", MAX_DROPS);
  if (s->n_drop > 0 && (!s->x0 || !s->y0 || !s->r0)) return fail(c, LBM_EINVAL, "droplet arrays missing");
  if (!(s->width > 0)) return fail(c, LBM_EINVAL, "interface width must be positive");
  std::vector<double> d(5 * (s->n_drop > 0 ? s->n_drop : 1), 0.0);
  for (int k = 0; k < s->n_drop; ++k) {
    d[5 * k] = s->x0[k]; d[5 * k + 1] = s->y0[k]; d[5 * k + 2] = s->r0[k];
    d[5 * k + 3] = s->ux0 ? s->ux0[k] : 0.0; d[5 * k + 4] = s->uy0 ? s->uy0[k] : 0.0;
  }
  const Layout& y = c->lay;
  CUDA_OK(c, cudaMemcpyAsync(c->ws + y.drops, d.data(), d.size() * 8, cudaMemcpyHostToDevice, c->stream));
  const double* dd = (const double*)(c->ws + y.drops);
  if (c->fp64) CUDA_OK(c, launch_init(c->Ld, dd, s->n_drop, s->width, c->eos.rho_g, c->eos.rho_l, c->stream));
  else CUDA_OK(c, launch_init(c->Lf, dd, s->n_drop, s->width, c->eos.rho_g, c->eos.rho_l, c->stream));
  CUDA_OK(c, cudaMemsetAsync(c->ws + y.step_ctr, 0, 16, c->stream));
  CUDA_OK(c, cudaMemsetAsync(c->ws + y.dm_ring, 0, (size_t)(DM_RING + 1) * 8, c->stream));
  CUDA_OK(c, cudaMemsetAsync(c->ws + y.carry, 0, (size_t)y.cap.bnodes * 8, c->stream));
  c->cur = 0;
  c->steps = 0;
  CUDA_OK(c, mass0_async(c));
  c->inited = true;
  c->rho_ok = false;
  c->tape.valid = false;
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int64_t n) {
  LBM_RANGE("lbm_step");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (n < 0) return fail(c, LBM_EINVAL, "negative step count");
  lbm_status s = c->fp64 ? do_step(c, c->Ld, n) : do_step(c, c->Lf, n);
  if (s == LBM_OK) c->steps += n;
  if (n > 0) c->tape.valid = false;
  return s;
}

lbm_status lbm_prepare_steps(lbm_ctx* c, int64_t n) {
  LBM_RANGE("lbm_prepare_steps");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (n < 0) return fail(c, LBM_EINVAL, "negative step count");
  return c->fp64 ? prepare_steps(c, c->Ld, n) : prepare_steps(c, c->Lf, n);
}

lbm_status lbm_set_collide_kernel(lbm_ctx* c, int32_t kind) {
  if (!c || !c->built) return LBM_ESTATE;
  if (kind < 0 || kind > 2)
    return fail(c, LBM_EINVAL, "collide kernel must be 0 (plain), 1 (TMA-pipelined) or 2 (column sweeps)");
  if (kind >= 1 && (c->fp64 || !c->tma_ok))
    return fail(c, LBM_EINVAL, "the TMA-pipelined collide kernel needs FP32 and the CUDA driver's tensor-map encoder");
  if (kind == 2 && (!sweep_shape(&c->cfg) || c->slab.on))
    return fail(c, LBM_EINVAL,
                "the column sweeps need the chemical-potential force with an equation of state, nx a multiple of 32 "
                "and ny of 8, and a whole lattice of two population lattices");
  if (kind == c->collide_kind) return LBM_OK;
  c->collide_kind = kind;
  // captured launches carry the old kernel: capture again
  for (auto& gr : c->graph)
    if (gr) { cudaGraphExecDestroy(gr); gr = nullptr; }
  for (auto& a : c->adj_graphs) cudaGraphExecDestroy(a.exec);
  c->adj_graphs.clear();
  refresh(c);
  return LBM_OK;
}

lbm_status lbm_set_spin_limit(lbm_ctx* c, int64_t polls) {
  if (!c || !c->built) return LBM_ESTATE;
  if (polls < 0) return fail(c, LBM_EINVAL, "negative spin limit");
  c->spin_limit = polls;
  for (auto& gr : c->graph)
    if (gr) { cudaGraphExecDestroy(gr); gr = nullptr; }
  for (auto& a : c->adj_graphs) cudaGraphExecDestroy(a.exec);
  c->adj_graphs.clear();
  refresh(c);
  return LBM_OK;
}

lbm_status lbm_set_mu_kernel(lbm_ctx* c, int32_t kind) {
  if (!c || !c->built) return LBM_ESTATE;
  if (kind < 0 || kind > 3) return fail(c, LBM_EINVAL, "chemical-potential kernel must be 0, 1, 2 or 3");
  if (kind >= 2 && c->fp64) return fail(c, LBM_EINVAL, "the row-sweep and fused chemical-potential kernels are FP32 only");
  if (kind == 3 && (c->cfg.force_model != LBM_FORCE_CHEMPOT || c->cfg.eos == LBM_EOS_NONE))
    return fail(c, LBM_EINVAL, "the fused chemical-potential kernel needs the chemical-potential force");
  if (kind == 3 && c->cfg.layout == LBM_LAYOUT_AA)
    return fail(c, LBM_EINVAL, "the fused chemical-potential kernel needs two population lattices");
  c->mu_kind = kind;
  c->rho_ok = false;   // a change to or from the fused pass moves where mu is kept
  if (kind == 3 && !c->near_built) {
    lbm_status st = near_list(c);
    if (st != LBM_OK) return st;
  }
  for (auto& gr : c->graph)
    if (gr) { cudaGraphExecDestroy(gr); gr = nullptr; }
  for (auto& a : c->adj_graphs) cudaGraphExecDestroy(a.exec);
  c->adj_graphs.clear();
  refresh(c);
  return LBM_OK;
}

lbm_status lbm_get_collide_kernel(lbm_ctx* c, int32_t* kind) {
  if (!c || !c->built || !kind) return LBM_ESTATE;
  // the kernel the step runs: the sweeps give way to kind 1 under the fused chemical-potential pass
  *kind = (c->fp64 || !c->tma_ok || c->collide_kind == 0) ? 0 : (step_sweeps(c->Lf, c->cur) ? 2 : 1);
  return LBM_OK;
}

lbm_status lbm_launches_per_step(lbm_ctx* c, int64_t* n) {
  if (!c || !c->built || !n) return LBM_ESTATE;
  *n = c->fp64 ? launches_per_step_overlap(c->Ld) : launches_per_step_overlap(c->Lf);
  return LBM_OK;
}

// The device address of page-locked host memory (which kernels can write directly), else null.
void* mapped_host(void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

lbm_status lbm_fields(lbm_ctx* c, void* rho, void* vx, void* vy, int32_t on_device) {
  LBM_RANGE("lbm_fields");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!rho || !vx || !vy) return fail(c, LBM_EINVAL, "null output");
  const long long dn = (long long)c->cfg.nx * c->cfg.ny;
  const size_t sz = c->lay.sz;
  if (!on_device) {
    // page-locked host arrays: the read-out kernel writes them directly, no staging copies
    void* hr = mapped_host(rho);
    void* hu = mapped_host(vx);
    void* hv = mapped_host(vy);
    if (hr && hu && hv) {
      if (c->fp64) CUDA_OK(c, launch_fields(c->Ld, c->cur, (double*)hr, (double*)hu, (double*)hv, c->stream));
      else CUDA_OK(c, launch_fields(c->Lf, c->cur, (float*)hr, (float*)hu, (float*)hv, c->stream));
      CUDA_OK(c, cudaStreamSynchronize(c->stream));
      return LBM_OK;
    }
  }
  char* stage = stage_area(c);
  char* r = on_device ? (char*)rho : stage;
  char* u = on_device ? (char*)vx : stage + dn * sz;
  char* v = on_device ? (char*)vy : stage + 2 * dn * sz;
  if (c->fp64) CUDA_OK(c, launch_fields(c->Ld, c->cur, (double*)r, (double*)u, (double*)v, c->stream));
  else CUDA_OK(c, launch_fields(c->Lf, c->cur, (float*)r, (float*)u, (float*)v, c->stream));
  if (!on_device) {
    CUDA_OK(c, cudaMemcpyAsync(rho, r, dn * sz, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaMemcpyAsync(vx, u, dn * sz, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaMemcpyAsync(vy, v, dn * sz, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

// ---- checkpoint / resume ------------------------------------------------------------------
namespace {

// CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), table-driven
uint32_t crc32_update(uint32_t crc, const unsigned char* p, size_t n) {
  static uint32_t table[256];
  static bool ready = false;
  if (!ready) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t v = i;
      for (int k = 0; k < 8; ++k) v = (v & 1u) ? (v >> 1) ^ 0xEDB88320u : v >> 1;
      table[i] = v;
    }
    ready = true;
  }
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xffu] ^ (crc >> 8);
  return ~crc;
}

// FNV-1a over the configuration's values (not its pointers), so a checkpoint is only loaded
// into a context that steps the same problem
uint64_t config_hash(const lbm_ctx* c) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  };
  const lbm_config& g = c->cfg;
  const int32_t ints[] = {g.nx, g.ny, g.walls, g.eos, g.coll, g.bc, g.precision, g.n_cyl, g.force_model};
  const double reals[] = {g.y_bottom, g.y_top, g.a, g.b, g.R, g.T_over_Tc, g.omega, g.k, g.kappa, g.tau,
                          g.s_e, g.s_eps, g.s_q, g.s_nu, g.gx, g.gy, c->rho_ref, g.dmu_w_walls};
  mix(ints, sizeof(ints));
  if (g.layout != LBM_LAYOUT_AB) mix(&g.layout, sizeof(g.layout));
  mix(reals, sizeof(reals));
  for (const std::vector<double>* v : {&c->cx, &c->cy, &c->r, &c->dmu}) mix(v->data(), v->size() * sizeof(double));
  return h;
}

struct CkptHeader {
  char magic[8];
  uint32_t version, precision;
  int32_t nx, ny, pitch, cur;
  uint64_t config_hash;
  int64_t steps;
  uint64_t n_bnodes;
  double mass0;
  uint64_t pop_bytes;
};
constexpr char CKPT_MAGIC[8] = {'L', 'B', 'M', 'G', 'B', 'C', 'K', '1'};
constexpr uint32_t CKPT_VERSION = 1;

}  // namespace

lbm_status lbm_save(lbm_ctx* c, const char* path) {
  LBM_RANGE("lbm_save");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!path) return fail(c, LBM_EINVAL, "null path");
  const Layout& y = c->lay;
  CkptHeader h{};
  std::memcpy(h.magic, CKPT_MAGIC, 8);
  h.version = CKPT_VERSION;
  h.precision = c->fp64 ? 1u : 0u;
  h.nx = c->cfg.nx; h.ny = c->cfg.ny; h.pitch = (int32_t)y.pitch; h.cur = c->cur;
  h.config_hash = config_hash(c);
  h.steps = c->steps;
  h.n_bnodes = (uint64_t)c->n_bnodes;
  lbm_status ms = resolve_mass0(c);
  if (ms != LBM_OK) return ms;
  // the steps queued on the context's stream finish before the state is copied out (the copies
  // below do not order themselves after a non-blocking stream)
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  h.mass0 = c->mass0;
  h.pop_bytes = 9ull * (uint64_t)y.plane * y.sz;
  const size_t ring_bytes = (size_t)(DM_RING + 1) * 8;
  std::vector<unsigned char> buf(sizeof(h) + h.pop_bytes + h.n_bnodes * 8 + ring_bytes + 8);
  unsigned char* p = buf.data();
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  CUDA_OK(c, cudaMemcpy(p, c->ws + (c->cur ? y.fB : y.fA), h.pop_bytes, cudaMemcpyDeviceToHost));
  p += h.pop_bytes;
  if (h.n_bnodes) CUDA_OK(c, cudaMemcpy(p, c->ws + y.carry, h.n_bnodes * 8, cudaMemcpyDeviceToHost));
  p += h.n_bnodes * 8;
  CUDA_OK(c, cudaMemcpy(p, c->ws + y.dm_ring, ring_bytes, cudaMemcpyDeviceToHost));
  p += ring_bytes;
  CUDA_OK(c, cudaMemcpy(p, c->ws + y.step_ctr, 8, cudaMemcpyDeviceToHost));
  const uint32_t crc = crc32_update(0u, buf.data(), buf.size());
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(c, LBM_EINVAL, "cannot open %s for writing", path);
  const bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size() && std::fwrite(&crc, 4, 1, f) == 1;
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) return fail(c, LBM_EINVAL, "writing %s failed", path);
  return LBM_OK;
}

lbm_status lbm_load(lbm_ctx* c, const char* path) {
  LBM_RANGE("lbm_load");
  if (!c || !c->built) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!path) return fail(c, LBM_EINVAL, "null path");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, LBM_EINVAL, "cannot open %s", path);
  std::vector<unsigned char> buf;
  unsigned char chunk[1 << 16];
  size_t got;
  while ((got = std::fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + got);
  const bool read_error = std::ferror(f) != 0;
  std::fclose(f);
  if (read_error) return fail(c, LBM_EINVAL, "reading %s failed", path);
  CkptHeader h{};
  if (buf.size() < sizeof(h) + 4) return fail(c, LBM_ECORRUPT, "%s is too short for a checkpoint", path);
  std::memcpy(&h, buf.data(), sizeof(h));
  if (std::memcmp(h.magic, CKPT_MAGIC, 8) != 0) return fail(c, LBM_ECORRUPT, "%s is not a checkpoint", path);
  if (h.version != CKPT_VERSION) return fail(c, LBM_ECORRUPT, "checkpoint format version %u", h.version);
  const size_t ring_bytes = (size_t)(DM_RING + 1) * 8;
  const uint64_t body = (uint64_t)sizeof(h) + h.pop_bytes + h.n_bnodes * 8 + ring_bytes + 8;
  if (h.pop_bytes > buf.size() || h.n_bnodes > buf.size() || buf.size() != body + 4)
    return fail(c, LBM_ECORRUPT, "%s is truncated or has trailing data", path);
  uint32_t crc;
  std::memcpy(&crc, buf.data() + body, 4);
  if (crc32_update(0u, buf.data(), (size_t)body) != crc) return fail(c, LBM_ECORRUPT, "%s fails its CRC-32", path);
  const Layout& y = c->lay;
  if (h.config_hash != config_hash(c) || h.nx != c->cfg.nx || h.ny != c->cfg.ny || h.pitch != (int32_t)y.pitch ||
      h.precision != (c->fp64 ? 1u : 0u) || h.n_bnodes != (uint64_t)c->n_bnodes ||
      h.pop_bytes != 9ull * (uint64_t)y.plane * y.sz || (h.cur != 0 && h.cur != 1))
    return fail(c, LBM_EINVAL, "%s is a checkpoint of another configuration", path);
  const unsigned char* p = buf.data() + sizeof(h);
  // on the context's stream, so that the steps queued after the load see the loaded state (a
  // copy on the default stream returns before its data has landed and is not ordered before a
  // non-blocking stream's work); finished before the host buffer goes
  CUDA_OK(c, cudaMemcpyAsync(c->ws + (h.cur ? y.fB : y.fA), p, h.pop_bytes, cudaMemcpyHostToDevice, c->stream));
  p += h.pop_bytes;
  if (h.n_bnodes) CUDA_OK(c, cudaMemcpyAsync(c->ws + y.carry, p, h.n_bnodes * 8, cudaMemcpyHostToDevice, c->stream));
  p += h.n_bnodes * 8;
  CUDA_OK(c, cudaMemcpyAsync(c->ws + y.dm_ring, p, ring_bytes, cudaMemcpyHostToDevice, c->stream));
  p += ring_bytes;
  CUDA_OK(c, cudaMemcpyAsync(c->ws + y.step_ctr, p, 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(c, cudaMemsetAsync(c->ws + y.kerr, 0, 16, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  c->cur = h.cur;
  c->steps = h.steps;
  c->mass0 = h.mass0;
  c->mass0_pending = false;
  c->inited = true;
  c->rho_ok = false;     // the next step forms the density and solid layers from the populations
  c->tape.valid = false;
  return LBM_OK;
}

lbm_status lbm_column_density(lbm_ctx* c, int32_t x, int32_t y0, int32_t n, double* out, int32_t on_device) {
  LBM_RANGE("lbm_column_density");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!out) return fail(c, LBM_EINVAL, "null output");
  if (x < 0 || x >= c->cfg.nx || y0 < 0 || n < 1 || (long long)y0 + n > c->cfg.ny)
    return fail(c, LBM_EINVAL, "column outside the lattice");
  double* d = on_device ? out : (double*)stage_area(c);
  if (c->fp64) CUDA_OK(c, launch_column(c->Ld, c->cur, x, y0, n, d, c->stream));
  else CUDA_OK(c, launch_column(c->Lf, c->cur, x, y0, n, d, c->stream));
  if (!on_device) {
    CUDA_OK(c, cudaMemcpyAsync(out, d, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

lbm_status lbm_max_speed(lbm_ctx* c, double* vmax) {
  LBM_RANGE("lbm_max_speed");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!vmax) return fail(c, LBM_EINVAL, "null output");
  auto* d = (unsigned long long*)stage_area(c);
  CUDA_OK(c, cudaMemsetAsync(d, 0, 8, c->stream));
  if (c->fp64) CUDA_OK(c, launch_max_speed(c->Ld, c->cur, d, c->stream));
  else CUDA_OK(c, launch_max_speed(c->Lf, c->cur, d, c->stream));
  CUDA_OK(c, cudaMemcpyAsync(vmax, d, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_populations(lbm_ctx* c, void* f, int32_t on_device) {
  LBM_RANGE("lbm_populations");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!f) return fail(c, LBM_EINVAL, "null output");
  const long long dn = (long long)c->cfg.nx * c->cfg.ny;
  const size_t sz = c->lay.sz;
  if (on_device) {
    if (c->fp64) CUDA_OK(c, launch_populations(c->Ld, c->cur, (double*)f, 0, 9, c->stream));
    else CUDA_OK(c, launch_populations(c->Lf, c->cur, (float*)f, 0, 9, c->stream));
    return LBM_OK;
  }
  // through the staging memory, as many planes at a time as it holds
  char* stage = stage_area(c);
  const int per = stage_planes(c);
  for (int i0 = 0; i0 < 9; i0 += per) {
    const int i1 = i0 + per < 9 ? i0 + per : 9;
    if (c->fp64) CUDA_OK(c, launch_populations(c->Ld, c->cur, (double*)stage, i0, i1, c->stream));
    else CUDA_OK(c, launch_populations(c->Lf, c->cur, (float*)stage, i0, i1, c->stream));
    CUDA_OK(c, cudaMemcpyAsync((char*)f + i0 * dn * sz, stage, (i1 - i0) * dn * sz, cudaMemcpyDeviceToHost, c->stream));
  }
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* c, const void* f, int32_t on_device) {
  LBM_RANGE("lbm_set_populations");
  if (!c || !c->built) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!f) return fail(c, LBM_EINVAL, "null input");
  const Layout& y = c->lay;
  const long long dn = (long long)c->cfg.nx * c->cfg.ny;
  c->cur = 0;
  if (on_device) {
    if (c->fp64) CUDA_OK(c, launch_set_populations(c->Ld, 0, (const double*)f, 0, 9, c->stream));
    else CUDA_OK(c, launch_set_populations(c->Lf, 0, (const float*)f, 0, 9, c->stream));
  } else {
    // through the staging memory (the second lattice, or one lattice's three staging planes)
    char* stage = c->ws + (c->cfg.layout == LBM_LAYOUT_AA ? y.stage : y.fB);
    const int per = stage_planes(c);
    for (int i0 = 0; i0 < 9; i0 += per) {
      const int i1 = i0 + per < 9 ? i0 + per : 9;
      CUDA_OK(c, cudaMemcpyAsync(stage, (const char*)f + i0 * dn * y.sz, (i1 - i0) * dn * y.sz,
                                 cudaMemcpyHostToDevice, c->stream));
      if (c->fp64) CUDA_OK(c, launch_set_populations(c->Ld, 0, (const double*)stage, i0, i1, c->stream));
      else CUDA_OK(c, launch_set_populations(c->Lf, 0, (const float*)stage, i0, i1, c->stream));
    }
  }
  CUDA_OK(c, cudaMemsetAsync(c->ws + y.step_ctr, 0, 16, c->stream));
  CUDA_OK(c, cudaMemsetAsync(c->ws + y.dm_ring, 0, (size_t)(DM_RING + 1) * 8, c->stream));
  CUDA_OK(c, cudaMemsetAsync(c->ws + y.carry, 0, (size_t)y.cap.bnodes * 8, c->stream));
  c->steps = 0;
  CUDA_OK(c, mass0_async(c));
  c->inited = true;
  c->rho_ok = false;
  c->tape.valid = false;
  return LBM_OK;
}

lbm_status lbm_mass(lbm_ctx* c, double* M, double* M0, double* dM_last) {
  LBM_RANGE("lbm_mass");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  const Layout& y = c->lay;
  if (c->fp64) CUDA_OK(c, launch_mass(c->Ld, c->cur, c->stream)); else CUDA_OK(c, launch_mass(c->Lf, c->cur, c->stream));
  double sc[2];
  unsigned long long ctr = 0;
  unsigned int kerr = 0;
  CUDA_OK(c, cudaMemcpyAsync(sc, c->ws + y.scalars, 16, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaMemcpyAsync(&ctr, c->ws + y.step_ctr, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaMemcpyAsync(&kerr, c->ws + y.kerr, 4, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  if (kerr != 0) {
    c->sticky = LBM_ETIMEOUT;
    return fail(c, LBM_ETIMEOUT, "a bounded wait of the pipelined collide kernel gave up");
  }
  double last = 0.0;
  if (ctr > 0)
    CUDA_OK(c, cudaMemcpy(&last, c->ws + y.dm_ring + ((ctr - 1) % DM_RING) * 8, 8, cudaMemcpyDeviceToHost));
  lbm_status ms = resolve_mass0(c);
  if (ms != LBM_OK) return ms;
  if (M) *M = sc[0] + (double)fluid_count(c) * c->rho_ref;
  if (M0) *M0 = c->mass0;
  if (dM_last) *dM_last = last;
  if (sc[1] != 0.0) return fail(c, LBM_EUNSTABLE, "%.0f non-finite populations", sc[1]);
  return LBM_OK;
}

lbm_status lbm_dM_history(lbm_ctx* c, double* out, int64_t n, int64_t* n_out) {
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  const Layout& y = c->lay;
  unsigned long long ctr = 0;
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  CUDA_OK(c, cudaMemcpy(&ctr, c->ws + y.step_ctr, 8, cudaMemcpyDeviceToHost));
  std::vector<double> ring(DM_RING);
  CUDA_OK(c, cudaMemcpy(ring.data(), c->ws + y.dm_ring, DM_RING * 8, cudaMemcpyDeviceToHost));
  long long avail = (long long)ctr < DM_RING ? (long long)ctr : DM_RING;
  long long k = n < avail ? n : avail;
  for (long long j = 0; j < k; ++j) out[j] = ring[(ctr - k + j) % DM_RING];
  if (n_out) *n_out = k;
  return LBM_OK;
}

lbm_status lbm_last_dM(lbm_ctx* c, double* dM) {
  if (!c || !c->inited || !dM) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  CUDA_OK(c, cudaMemcpyAsync(dM, c->ws + c->lay.dm_ring + (size_t)DM_RING * 8, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_last_dM_async(lbm_ctx* c, double* dM) {
  if (!c || !c->inited || !dM) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  const double* src = reinterpret_cast<const double*>(c->ws + c->lay.dm_ring + (size_t)DM_RING * 8);
  // page-locked host memory: one thread stores the value into it (a copy-engine copy between
  // two steps would hold the next step back for its own latency); other memory: a copy
  if (void* dst = mapped_host(dM)) {
    CUDA_OK(c, launch_copy8(src, static_cast<double*>(dst), c->stream));
    return LBM_OK;
  }
  CUDA_OK(c, cudaMemcpyAsync(dM, src, 8, cudaMemcpyDeviceToHost, c->stream));
  return LBM_OK;
}

lbm_status lbm_profile_steps(lbm_ctx* c, int64_t n, double* ms5) {
  LBM_RANGE("lbm_profile_steps");
  if (!c || !c->inited || !ms5) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  return c->fp64 ? profile_steps(c, c->Ld, n, ms5) : profile_steps(c, c->Lf, n, ms5);
}

lbm_status lbm_eos_info(lbm_ctx* c, double* o) {
  if (!c || !o) return LBM_EINVAL;
  o[0] = c->eos.Tc; o[1] = c->eos.rho_c; o[2] = c->eos.T; o[3] = c->eos.alpha;
  o[4] = c->eos.rho_g; o[5] = c->eos.rho_l; o[6] = c->eos.mu_sat; o[7] = c->eos.p_sat;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  for (auto& g : c->graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto& a : c->adj_graphs) cudaGraphExecDestroy(a.exec);
  for (cudaEvent_t e : {c->ev_start, c->ev_rec[0], c->ev_rec[1], c->ev_rev[0], c->ev_rev[1], c->ev_fork, c->ev_join})
    if (e) cudaEventDestroy(e);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Batched lattices
// ---------------------------------------------------------------------------------------
struct lbm_batch {
  int n = 0;
  bool fp64 = false;
  std::vector<lbm_ctx*> ctx;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  std::vector<size_t> inst_off, inst_bytes;
  size_t tab_off = 0;
  // table offsets inside the tables region
  size_t t_lat = 0, t_tiles = 0, t_s1 = 0, t_s2 = 0, t_bc = 0, t_first = 0, t_group = 0, t_part = 0, t_bar = 0,
         t_err = 0;
  int groups = 2;
  long long cap_tiles = 0, cap_s1 = 0, cap_s2 = 0, cap_bc = 0;
  BatchDev dev{};
  bool tables = false;
  int grid = 0;
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  long long graph_steps = -1;
  int graph_cur = -1;
  long long spin_limit = 1LL << 22;
  int tile_log2w = BATCH_TILE_LOG2W_DEFAULT;
  int cur = 0;
  std::string err;
};

namespace {

struct BatchPlan {
  std::vector<size_t> off, bytes;
  size_t tab_off, total;
  size_t t_lat, t_tiles, t_s1, t_s2, t_bc, t_first, t_group, t_part, t_bar, t_err;
  long long cap_tiles, cap_s1, cap_s2, cap_bc;
};

lbm_status plan_batch(int n, const lbm_config* cfgs, BatchPlan* P, char* msg) {
  if (n < 1 || !cfgs) { std::snprintf(msg, 256, "batch needs at least one configuration"); return LBM_EINVAL; }
  P->off.resize(n);
  P->bytes.resize(n);
  size_t o = 0;
  P->cap_tiles = P->cap_s1 = P->cap_s2 = P->cap_bc = 0;
  for (int k = 0; k < n; ++k) {
    lbm_status s = validate(&cfgs[k], msg);
    if (s != LBM_OK) return s;
    if (cfgs[k].precision != cfgs[0].precision) { std::snprintf(msg, 256, "all instances of a batch share one precision"); return LBM_EINVAL; }
    if (cfgs[k].force_model != LBM_FORCE_CHEMPOT) { std::snprintf(msg, 256, "the batched kernel runs the chemical-potential force only"); return LBM_EINVAL; }
    Layout L = make_layout(&cfgs[k]);
    P->off[k] = o;
    P->bytes[k] = L.total;
    o = align_up(o + L.total);
    const int bb = batch_block_size();
    long long most = 0;   // room for the tile list of any shape
    for (int lw = BATCH_TILE_LOG2W_MIN; lw <= BATCH_TILE_LOG2W_MAX; ++lw) {
      const long long t = batch_node_tiles(cfgs[k].nx, cfgs[k].ny, lw);
      most = t > most ? t : most;
    }
    P->cap_tiles += most;
    P->cap_s1 += (L.cap.s1 + bb - 1) / bb;
    // one lattice in AA order: the boundary nodes' moments are saved in the second solid layer's
    // phase, in chunks that follow the layer's own
    P->cap_s2 += (L.cap.s2 + bb - 1) / bb + (cfgs[k].layout == LBM_LAYOUT_AA ? (L.cap.bnodes + bb - 1) / bb : 0);
    P->cap_bc += (L.cap.bnodes + bb - 1) / bb;
  }
  P->tab_off = o;
  size_t t = 0;
  auto take = [&](size_t bytes) { size_t at = t; t = align_up(t + bytes); return at; };
  const size_t lat_sz = cfgs[0].precision == LBM_FP64 ? sizeof(Lattice<double>) : sizeof(Lattice<float>);
  P->t_lat = take((size_t)n * lat_sz);
  P->t_tiles = take((size_t)P->cap_tiles * sizeof(int2));
  P->t_s1 = take((size_t)(P->cap_s1 + 1) * sizeof(int2));
  P->t_s2 = take((size_t)(P->cap_s2 + 1) * sizeof(int2));
  P->t_bc = take((size_t)(P->cap_bc + 1) * sizeof(int2));
  P->t_first = take((size_t)n * sizeof(int2));
  P->t_group = take((size_t)n);
  P->t_part = take((size_t)(P->cap_bc + 1) * sizeof(double));
  P->t_bar = take(16 + BATCH_WORK_COUNTERS * 8);   // barrier words, then the work counters
  P->t_err = take(16);
  P->total = P->tab_off + t;
  return LBM_OK;
}

lbm_status bfail(lbm_batch* b, lbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  return s;
}

#define BCUDA(b, call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return bfail(b, LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename real>
lbm_status batch_tables(lbm_batch* b) {
  const int bb = batch_block_size();
  const int G = b->groups;
  std::vector<Lattice<real>> lats(b->n);
  // groups of about equal node counts: largest instances first, each to the lighter group
  std::vector<uint8_t> group(b->n, 0);
  if (G == 2) {
    std::vector<int> order(b->n);
    for (int k = 0; k < b->n; ++k) order[k] = k;
    auto nodes = [&](int k) { return (long long)b->ctx[k]->cfg.nx * b->ctx[k]->cfg.ny; };
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return nodes(u) > nodes(v); });
    long long load[2] = {0, 0};
    for (int k : order) {
      const int g = load[1] < load[0] ? 1 : 0;
      group[k] = (uint8_t)g;
      load[g] += nodes(k);
    }
  }
  std::vector<int2> tiles, s1, s2, bc, inst_bc(b->n);
  BatchDev& d = b->dev;
  for (int g = 0; g < 2; ++g) {
    d.tile_start[g] = (int)tiles.size();
    d.s1_start[g] = (int)s1.size();
    d.s2_start[g] = (int)s2.size();
    d.bc_start[g] = (int)bc.size();
    for (int k = 0; k < b->n; ++k) {
      if (group[k] != g) continue;
      const Lattice<real>& L = b->fp64 ? *reinterpret_cast<const Lattice<real>*>(&b->ctx[k]->Ld)
                                       : *reinterpret_cast<const Lattice<real>*>(&b->ctx[k]->Lf);
      lats[k] = L;
      const long long nt = batch_node_tiles(L.nx, L.ny, b->tile_log2w);
      for (long long t = 0; t < nt; ++t) tiles.push_back(make_int2(k, (int)t));
      for (int j = 0; j < L.n_s1; j += bb) s1.push_back(make_int2(k, j));
      for (int j = 0; j < L.n_s2; j += bb) s2.push_back(make_int2(k, j));
      if (L.aa)
        for (int j = 0; j < L.n_bnodes; j += bb) s2.push_back(make_int2(k, j | BATCH_BMOM_ITEM));
      inst_bc[k].x = (int)bc.size();
      for (int j = 0; j < L.n_bnodes; j += bb) bc.push_back(make_int2(k, j));
      inst_bc[k].y = (int)bc.size();
    }
  }
  d.tile_start[2] = (int)tiles.size();
  d.s1_start[2] = (int)s1.size();
  d.s2_start[2] = (int)s2.size();
  d.bc_start[2] = (int)bc.size();
  if ((long long)tiles.size() > b->cap_tiles || (long long)s1.size() > b->cap_s1 + 1 ||
      (long long)s2.size() > b->cap_s2 + 1 || (long long)bc.size() > b->cap_bc + 1)
    return bfail(b, LBM_ENOMEM, "batch work lists exceed their capacity");
  char* t = b->ws + b->tab_off;
  BCUDA(b, cudaMemcpyAsync(t + b->t_lat, lats.data(), lats.size() * sizeof(Lattice<real>), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(t + b->t_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  if (!s1.empty()) BCUDA(b, cudaMemcpyAsync(t + b->t_s1, s1.data(), s1.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  if (!s2.empty()) BCUDA(b, cudaMemcpyAsync(t + b->t_s2, s2.data(), s2.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  if (!bc.empty()) BCUDA(b, cudaMemcpyAsync(t + b->t_bc, bc.data(), bc.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(t + b->t_first, inst_bc.data(), inst_bc.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(t + b->t_group, group.data(), group.size(), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemsetAsync(t + b->t_err, 0, 16, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  d.n_inst = b->n;
  d.groups = G;
  d.lat = t + b->t_lat;
  d.inst_group = (const uint8_t*)(t + b->t_group);
  d.tile_log2w = b->tile_log2w;
  d.node_tiles = (const int2*)(t + b->t_tiles);
  d.s1_items = (const int2*)(t + b->t_s1);
  d.s2_items = (const int2*)(t + b->t_s2);
  d.bc_items = (const int2*)(t + b->t_bc);
  d.inst_bc = (const int2*)(t + b->t_first);
  d.bc_partials = (double*)(t + b->t_part);
  d.bar = (unsigned int*)(t + b->t_bar);
  d.work = (unsigned long long*)(t + b->t_bar + 16);
  d.err = (int*)(t + b->t_err);
  d.spin_limit = b->spin_limit;
  b->grid = batch_grid_size(b->fp64);
  b->tables = true;
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_workspace_size(int32_t n, const lbm_config* cfgs, size_t* bytes) {
  if (!bytes) return LBM_EINVAL;
  BatchPlan P;
  char msg[256];
  lbm_status s = plan_batch(n, cfgs, &P, msg);
  if (s != LBM_OK) return s;
  *bytes = P.total;
  return LBM_OK;
}

lbm_status lbm_batch_create(int32_t n, const lbm_config* cfgs, void* stream, void* workspace, size_t bytes,
                            lbm_batch** out) {
  LBM_RANGE("lbm_batch_create");
  if (!out) return LBM_EINVAL;
  lbm_batch* b = new lbm_batch();
  *out = b;
  BatchPlan P;
  char msg[256] = {0};
  lbm_status s = plan_batch(n, cfgs, &P, msg);
  if (s != LBM_OK) { b->err = msg; return s; }
  if (!workspace || ((uintptr_t)workspace) % ALIGN) return bfail(b, LBM_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (bytes < P.total) return bfail(b, LBM_ENOMEM, "batch workspace of %zu bytes, %zu needed", bytes, P.total);
  b->n = n;
  b->fp64 = cfgs[0].precision == LBM_FP64;
  b->stream = (cudaStream_t)stream;
  b->ws = (char*)workspace;
  b->inst_off = P.off;
  b->inst_bytes = P.bytes;
  b->tab_off = P.tab_off;
  b->t_lat = P.t_lat; b->t_tiles = P.t_tiles; b->t_s1 = P.t_s1; b->t_s2 = P.t_s2; b->t_bc = P.t_bc;
  b->t_first = P.t_first; b->t_group = P.t_group; b->t_part = P.t_part; b->t_bar = P.t_bar; b->t_err = P.t_err;
  b->cap_tiles = P.cap_tiles; b->cap_s1 = P.cap_s1; b->cap_s2 = P.cap_s2; b->cap_bc = P.cap_bc;
  b->ctx.assign(n, nullptr);
  for (int k = 0; k < n; ++k) {
    lbm_status st = lbm_create(&cfgs[k], stream, b->ws + P.off[k], P.bytes[k], &b->ctx[k]);
    if (st != LBM_OK) return bfail(b, st, "instance %d: %s", k, b->ctx[k] ? b->ctx[k]->err.c_str() : "");
  }
  return LBM_OK;
}

lbm_status lbm_batch_build_links(lbm_batch* b) {
  LBM_RANGE("lbm_batch_build_links");
  if (!b || b->ctx.empty()) return LBM_ESTATE;
  for (int k = 0; k < b->n; ++k) {
    lbm_status st = lbm_build_links(b->ctx[k]);
    if (st != LBM_OK) return bfail(b, st, "instance %d: %s", k, b->ctx[k]->err.c_str());
  }
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  return b->fp64 ? batch_tables<double>(b) : batch_tables<float>(b);
}

lbm_status lbm_batch_init(lbm_batch* b, const lbm_init_spec* specs) {
  LBM_RANGE("lbm_batch_init");
  if (!b || !b->tables || !specs) return LBM_ESTATE;
  for (int k = 0; k < b->n; ++k) {
    lbm_status st = lbm_init(b->ctx[k], &specs[k]);
    if (st != LBM_OK) return bfail(b, st, "instance %d: %s", k, b->ctx[k]->err.c_str());
  }
  b->cur = 0;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n) {
  LBM_RANGE("lbm_batch_step");
  if (!b || !b->tables) return LBM_ESTATE;
  for (int k = 0; k < b->n; ++k) {
    if (!b->ctx[k]->inited) return bfail(b, LBM_ESTATE, "instance %d not initialised", k);
    if (b->ctx[k]->cur != b->cur) return bfail(b, LBM_ESTATE, "instance %d was stepped on its own", k);
  }
  if (n <= 0) return n == 0 ? LBM_OK : LBM_EINVAL;
  if (n > (1LL << 30)) return bfail(b, LBM_EINVAL, "too many steps in one launch");
  b->dev.spin_limit = b->spin_limit;
  if (b->use_graph && (b->graph_steps != n || b->graph_cur != b->cur || !b->graph)) {
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = launch_batch(b->dev, b->fp64, b->grid, (int)n, b->cur, b->stream);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      e = e1 != cudaSuccess ? e1 : e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) {
      // a cooperative launch that cannot be captured is issued directly instead
      cudaGetLastError();
      b->use_graph = false;
      b->graph = nullptr;
    } else {
      b->graph_steps = n;
      b->graph_cur = b->cur;
    }
  }
  if (b->use_graph && b->graph) BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  else BCUDA(b, launch_batch(b->dev, b->fp64, b->grid, (int)n, b->cur, b->stream));
  const int flip = (int)(n & 1);
  b->cur ^= flip;
  for (int k = 0; k < b->n; ++k) {
    b->ctx[k]->cur ^= flip;
    b->ctx[k]->steps += n;
    b->ctx[k]->rho_ok = false;
  }
  return LBM_OK;
}

lbm_status lbm_batch_check(lbm_batch* b) {
  if (!b || !b->tables) return LBM_ESTATE;
  int e = 0;
  BCUDA(b, cudaMemcpyAsync(&e, b->dev.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  if (e) return bfail(b, LBM_ETIMEOUT, "a grid barrier wait gave up");
  return LBM_OK;
}

lbm_status lbm_batch_set_spin_limit(lbm_batch* b, int64_t polls) {
  if (!b || polls < 0) return LBM_EINVAL;
  b->spin_limit = polls;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  b->graph_steps = -1;
  if (b->tables) {
    BCUDA(b, cudaMemsetAsync(b->dev.err, 0, sizeof(int), b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
  }
  return LBM_OK;
}

lbm_status lbm_batch_set_tile(lbm_batch* b, int32_t log2w) {
  if (!b || b->ctx.empty()) return LBM_ESTATE;
  if (log2w < BATCH_TILE_LOG2W_MIN || log2w > BATCH_TILE_LOG2W_MAX)
    return bfail(b, LBM_EINVAL, "tile width 2^%d outside 2^%d .. 2^%d", log2w, BATCH_TILE_LOG2W_MIN,
                 BATCH_TILE_LOG2W_MAX);
  b->tile_log2w = log2w;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  b->graph_steps = -1;
  if (!b->tables) return LBM_OK;
  return b->fp64 ? batch_tables<double>(b) : batch_tables<float>(b);
}

lbm_status lbm_batch_set_schedule(lbm_batch* b, int32_t groups) {
  if (!b || b->ctx.empty()) return LBM_ESTATE;
  if (groups != 1 && groups != 2) return bfail(b, LBM_EINVAL, "groups must be 1 or 2, not %d", groups);
  b->groups = groups;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  b->graph_steps = -1;
  if (!b->tables) return LBM_OK;
  return b->fp64 ? batch_tables<double>(b) : batch_tables<float>(b);
}

namespace {
// device time (ms) of `steps` steps of the batch as it is set up, after one untimed launch of
// the same length (which also captures its graph)
lbm_status time_batch(lbm_batch* b, int64_t steps, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  lbm_status st = lbm_batch_step(b, steps);
  if (st != LBM_OK) return st;
  cudaEventRecord(e0, b->stream);
  st = lbm_batch_step(b, steps);
  cudaEventRecord(e1, b->stream);
  if (st != LBM_OK) return st;
  st = lbm_batch_check(b);
  if (st == LBM_OK && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) st = bfail(b, LBM_ECUDA, "event timing failed");
  return st;
}
}  // namespace

lbm_status lbm_batch_autotune(lbm_batch* b, int64_t steps, int32_t* chosen_log2w, int32_t* chosen_groups,
                              double* ms) {
  LBM_RANGE("lbm_batch_autotune");
  if (!b || !b->tables) return LBM_ESTATE;
  if (steps < 1 || steps > (1LL << 20)) return bfail(b, LBM_EINVAL, "trial steps must lie in [1, 2^20]");
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  int best = b->tile_log2w, best_g = b->groups;
  double best_ms = 1e300;
  lbm_status st = LBM_OK;
  // tile shapes under the current schedule, then both schedules with the fastest shape
  for (int lw = BATCH_TILE_LOG2W_MIN; lw <= BATCH_TILE_LOG2W_MAX && st == LBM_OK; ++lw) {
    float t = 0.f;
    st = lbm_batch_set_tile(b, lw);
    if (st == LBM_OK) st = time_batch(b, steps, e0, e1, &t);
    if (ms) ms[lw - BATCH_TILE_LOG2W_MIN] = t;
    if (st == LBM_OK && t < best_ms) { best_ms = t; best = lw; }
  }
  if (st == LBM_OK) st = lbm_batch_set_tile(b, best);
  best_ms = 1e300;
  for (int g = 1; g <= 2 && st == LBM_OK; ++g) {
    float t = 0.f;
    st = lbm_batch_set_schedule(b, g);
    if (st == LBM_OK) st = time_batch(b, steps, e0, e1, &t);
    if (ms) ms[5 + g - 1] = t;
    if (st == LBM_OK && t < best_ms) { best_ms = t; best_g = g; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LBM_OK) return st;
  if (chosen_log2w) *chosen_log2w = best;
  if (chosen_groups) *chosen_groups = best_g;
  return lbm_batch_set_schedule(b, best_g);
}

lbm_status lbm_batch_instance(lbm_batch* b, int32_t k, lbm_ctx** ctx) {
  if (!b || !ctx || k < 0 || k >= b->n) return LBM_EINVAL;
  *ctx = b->ctx[k];
  return LBM_OK;
}

lbm_status lbm_batch_info(lbm_batch* b, int64_t* out4) {
  if (!b || !out4) return LBM_EINVAL;
  out4[0] = b->grid;
  out4[1] = b->dev.tile_start[2];
  out4[2] = b->use_graph ? 1 : 0;
  out4[3] = b->dev.bc_start[2];
  return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : "null batch"; }

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto* c : b->ctx) lbm_destroy(c);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Objective and reverse mode
// ---------------------------------------------------------------------------------------
namespace {

// Adjoint workspace: checkpoints of the populations and of the Eq. 18 carries at the start of
// every segment of `every` steps; two sets of segment buffers -- the states of one segment
// (its checkpoint copied to slot 0, the k recomputed ones in slots 1..k) with the density and
// chemical-potential planes of each of its steps; the adjoint planes; and the snapshots that
// restore the forward state afterwards.
struct AdjLayout {
  long long n, every, nseg;
  size_t ckpt, ckcarry, seg, segrho, segmu, lam0, lam1, lam_bc, lrj, lamF, Lmu, Lrho, bct, ring, ctr, carry, grad;
  size_t state;   // bytes of one population lattice (9 planes)
  size_t total;
};

AdjLayout make_adj_layout(const lbm_ctx* c, long long n, long long every) {
  AdjLayout A{};
  const Layout& y = c->lay;
  if (every <= 0) every = (long long)std::ceil(std::sqrt((double)n));
  if (every < 1) every = 1;
  if (every > n) every = n;
  A.n = n;
  A.every = every;
  A.nseg = (n + every - 1) / every;
  A.state = align_up(9 * (size_t)y.plane * y.sz);
  const size_t pl = (size_t)y.plane * y.sz;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
  A.ckpt = take((size_t)A.nseg * A.state);
  A.ckcarry = take((size_t)A.nseg * (size_t)y.cap.bnodes * 8);
  // two sets of segment buffers: one is recomputed while the other is swept backwards
  A.seg = take(2 * (size_t)(every + 1) * A.state);
  A.segrho = take(2 * (size_t)every * pl);
  A.segmu = take(2 * (size_t)every * pl);
  A.lam0 = take(9 * pl);
  A.lam1 = take(9 * pl);
  A.lam_bc = take(9 * pl);
  A.lrj = take(3 * pl);
  A.lamF = take(2 * pl);
  A.Lmu = take(pl);
  A.Lrho = take(pl);
  A.bct = take((size_t)y.plane);
  A.ring = take((size_t)(DM_RING + 1) * 8);
  A.ctr = take(16);
  A.carry = take((size_t)y.cap.bnodes * 8);
  A.grad = take((size_t)(3 * c->cfg.n_cyl + 1) * 8);
  A.total = o;
  return A;
}

template <typename real>
lbm_status forward_checkpointed(lbm_ctx* c, const Lattice<real>& L, const AdjLayout& A) {
  const Layout& y = c->lay;
  char* w = c->tape.ws;
  for (long long s = 0; s < A.nseg; ++s) {
    const long long k = s + 1 < A.nseg ? A.every : A.n - s * A.every;
    CUDA_OK(c, cudaMemcpyAsync(w + A.ckpt + s * A.state, L.f[c->cur], 9 * (size_t)y.plane * y.sz,
                               cudaMemcpyDeviceToDevice, c->stream));
    if (c->n_bnodes > 0)
      CUDA_OK(c, cudaMemcpyAsync(w + A.ckcarry + s * (size_t)y.cap.bnodes * 8, L.carry, (size_t)c->n_bnodes * 8,
                                 cudaMemcpyDeviceToDevice, c->stream));
    lbm_status st = do_step(c, L, k);
    if (st != LBM_OK) return st;
    c->steps += k;
  }
  return LBM_OK;
}

template <typename real>
lbm_status objective(lbm_ctx* c, const Lattice<real>& L, int body, double* J, void* seed, int on_device) {
  const Layout& y = c->lay;
  // the lattice that the next step overwrites completely holds the scratch
  char* stage = c->ws + (c->cur ? y.fA : y.fB);
  // touch flags, 4 partial sums per block and the seed fit in the 9 planes for any plane size
  const size_t nred = 4 * (size_t)objective_blocks(y.plane);
  uint8_t* touch = (uint8_t*)stage;
  double* red = (double*)(stage + align_up((size_t)y.plane));
  real* out = (real*)(stage + align_up((size_t)y.plane) + align_up(nred * 8));
  CUDA_OK(c, objective_sums(L, c->cur, body, touch, red, c->eos.rho_g, c->eos.rho_l, c->stream));
  std::vector<double> part(nred);
  CUDA_OK(c, cudaMemcpyAsync(part.data(), red, nred * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  double h[4] = {0, 0, 0, 0};
  for (size_t b = 0; b < nred; b += 4)
    for (int k = 0; k < 4; ++k) h[k] += part[b + k];
  if (!(h[0] != 0.0)) return fail(c, LBM_EINVAL, "no excess density: the objective is undefined");
  const double y_cm = h[1] / h[0];
  const double dphi = c->eos.rho_l - c->eos.rho_g;
  const double arc = h[3] > 0 ? 2.0 * M_PI * c->r[body] / h[3] : 0.0;
  *J = y_cm + arc * h[2];
  if (seed) {
    const long long dn = (long long)c->cfg.nx * c->cfg.ny;
    real* dst = on_device ? (real*)seed : out;
    CUDA_OK(c, objective_seed(L, touch, y_cm, h[0], arc / dphi, dst, c->stream));
    if (!on_device) {
      CUDA_OK(c, cudaMemcpyAsync(seed, dst, dn * y.sz, cudaMemcpyDeviceToHost, c->stream));
      CUDA_OK(c, cudaStreamSynchronize(c->stream));
    }
  }
  return LBM_OK;
}

template <typename real>
lbm_status adjoint(lbm_ctx* c, const Lattice<real>& L, const void* drho, const void* df, int on_device, double* grad,
                   void* df0) {
  const Layout& y = c->lay;
  const AdjLayout A = make_adj_layout(c, c->tape.n, c->tape.every);
  char* w = c->tape.ws;
  cudaStream_t st = c->stream;
  const long long dn = (long long)c->cfg.nx * c->cfg.ny;
  const size_t pl = (size_t)y.plane * y.sz;
  // snapshots of the forward state that the recomputation overwrites
  CUDA_OK(c, cudaMemcpyAsync(w + A.ring, L.dM_ring, (size_t)(DM_RING + 1) * 8, cudaMemcpyDeviceToDevice, st));
  CUDA_OK(c, cudaMemcpyAsync(w + A.ctr, L.step_ctr, 8, cudaMemcpyDeviceToDevice, st));
  if (c->n_bnodes > 0)
    CUDA_OK(c, cudaMemcpyAsync(w + A.carry, L.carry, (size_t)c->n_bnodes * 8, cudaMemcpyDeviceToDevice, st));
  // seeds (host seeds are staged in planes that are overwritten before they are read)
  const real* s_rho = (const real*)drho;
  const real* s_f = (const real*)df;
  if (!on_device) {
    if (drho) {
      CUDA_OK(c, cudaMemcpyAsync(w + A.Lmu, drho, dn * y.sz, cudaMemcpyHostToDevice, st));
      s_rho = (const real*)(w + A.Lmu);
    }
    if (df) {
      CUDA_OK(c, cudaMemcpyAsync(w + A.lam_bc, df, 9 * dn * y.sz, cudaMemcpyHostToDevice, st));
      s_f = (const real*)(w + A.lam_bc);
    }
  }
  real* lam[2] = {(real*)(w + A.lam0), (real*)(w + A.lam1)};
  CUDA_OK(c, adj_seed(L, lam[0], s_rho, s_f, st));
  CUDA_OK(c, cudaMemsetAsync(lam[1], 0, 9 * pl, st));
  CUDA_OK(c, cudaMemsetAsync(w + A.lam_bc, 0, 9 * pl, st));
  CUDA_OK(c, cudaMemsetAsync(w + A.lamF, 0, 2 * pl, st));
  CUDA_OK(c, cudaMemsetAsync(w + A.grad, 0, (size_t)(3 * c->cfg.n_cyl + 1) * 8, st));
  CUDA_OK(c, adj_flags(L, (uint8_t*)(w + A.bct), st));
  AdjBuffers B{};
  B.lam_bc = w + A.lam_bc;
  B.lrj = w + A.lrj;
  B.lamF = w + A.lamF;
  B.Lmu = w + A.Lmu;
  B.Lrho = w + A.Lrho;
  B.bct = (const uint8_t*)(w + A.bct);
  B.grad = (double*)(w + A.grad);
  B.n_cyl = c->cfg.n_cyl;
  // Pipeline: the recomputation of segment s-1 (second stream) overlaps the reverse steps of
  // segment s (the context's stream); the two use alternate buffer sets.  Events order each
  // buffer's reuse: a set is recomputed only after the reverse steps that read it are done.
  if (!c->aux) {
    CUDA_OK(c, cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&c->ev_start, &c->ev_rec[0], &c->ev_rec[1], &c->ev_rev[0], &c->ev_rev[1]})
      CUDA_OK(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  cudaStream_t aux = c->aux;
  auto seg_at = [&](int buf, long long i) { return w + A.seg + ((size_t)buf * (A.every + 1) + i) * A.state; };
  auto rho_at = [&](int buf, long long i) { return w + A.segrho + ((size_t)buf * A.every + i) * pl; };
  auto mu_at = [&](int buf, long long i) { return w + A.segmu + ((size_t)buf * A.every + i) * pl; };
  auto seg_len = [&](long long s) { return s + 1 < A.nseg ? A.every : A.n - s * A.every; };
  // the chemical potential of the solid layers is constant: every step's plane starts as a
  // copy of the lattice's own plane, whose fluid values the recomputation overwrites
  for (int buf = 0; buf < 2; ++buf)
    for (long long i = 0; i < A.every; ++i)
      CUDA_OK(c, cudaMemcpyAsync(mu_at(buf, i), L.mu, pl, cudaMemcpyDeviceToDevice, st));
  CUDA_OK(c, cudaMemsetAsync(w + A.Lrho, 0, pl, st));

  // the graphs the sweep needs, captured before any of them runs
  auto find = [&](int kind, int buf, long long k, int par) -> cudaGraphExec_t {
    for (auto& a : c->adj_graphs)
      if (a.ws == w && a.n == A.n && a.every == A.every && a.kind == kind && a.buf == buf && a.k == k &&
          a.parity == par)
        return a.exec;
    return nullptr;
  };
  auto capture = [&](int kind, int buf, long long k, int par) -> lbm_status {
    if (find(kind, buf, k, par)) return LBM_OK;
    cudaGraph_t gr;
    CUDA_OK(c, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    Lattice<real> Lc = L;
    auto at = [&](long long i) {
      Lc.f[0] = (real*)seg_at(buf, i);
      Lc.f[1] = (real*)seg_at(buf, i + 1);
      Lc.rho = (real*)rho_at(buf, i);
      Lc.mu = (real*)mu_at(buf, i);
      Lc.psip = nullptr;   // the recomputation evaluates psi' in its own chemical-potential pass
    };
    if (kind == 0) {
      // the segment's states (and each step's rho, mu) from slot 0
      for (long long i = 0; i < k && e == cudaSuccess; ++i) {
        at(i);
        e = launch_step(Lc, 0, st);
      }
    } else {
      // its reverse steps: step i reads f^i from slot i and the values its links used from
      // slot i+1
      int pp = par;
      for (long long i = k - 1; i >= 0 && e == cudaSuccess; --i) {
        at(i);
        AdjBuffers Bi = B;
        Bi.lam_in = lam[pp];
        Bi.lam_out = lam[pp ^ 1];
        e = adj_step(Lc, Bi, st);
        pp ^= 1;
      }
    }
    cudaError_t e2 = cudaStreamEndCapture(st, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess)
      return fail(c, LBM_ECUDA, "reverse-sweep capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    cudaGraphExec_t g = nullptr;
    cudaError_t e3 = cudaGraphInstantiate(&g, gr, 0);
    cudaGraphDestroy(gr);
    if (e3 != cudaSuccess) return fail(c, LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e3));
    c->adj_graphs.push_back({w, A.n, A.every, k, kind, buf, par, g});
    return LBM_OK;
  };
  {
    int p = 0;
    for (long long s = A.nseg - 1; s >= 0; --s) {
      const long long k = seg_len(s);
      lbm_status r1 = capture(0, (int)(s & 1), k, 0);
      if (r1 != LBM_OK) return r1;
      lbm_status r2 = capture(1, (int)(s & 1), k, p);
      if (r2 != LBM_OK) return r2;
      p ^= (int)(k & 1);
    }
  }
  // recomputation of segment s into buffer set s & 1, on the second stream
  auto recompute = [&](long long s) -> lbm_status {
    const int buf = (int)(s & 1);
    CUDA_OK(c, cudaMemcpyAsync(seg_at(buf, 0), w + A.ckpt + s * A.state, 9 * pl, cudaMemcpyDeviceToDevice, aux));
    if (c->n_bnodes > 0)
      CUDA_OK(c, cudaMemcpyAsync(L.carry, w + A.ckcarry + s * (size_t)y.cap.bnodes * 8, (size_t)c->n_bnodes * 8,
                                 cudaMemcpyDeviceToDevice, aux));
    CUDA_OK(c, cudaGraphLaunch(find(0, buf, seg_len(s), 0), aux));
    CUDA_OK(c, cudaEventRecord(c->ev_rec[buf], aux));
    return LBM_OK;
  };
  CUDA_OK(c, cudaEventRecord(c->ev_start, st));
  CUDA_OK(c, cudaStreamWaitEvent(aux, c->ev_start, 0));
  lbm_status rs = recompute(A.nseg - 1);
  if (rs != LBM_OK) return rs;
  int p = 0;
  for (long long s = A.nseg - 1; s >= 0; --s) {
    const int buf = (int)(s & 1);
    const long long k = seg_len(s);
    if (s >= 1) {
      // buffer set buf^1 was last read by the reverse steps of segment s+1
      if (s + 1 < A.nseg) CUDA_OK(c, cudaStreamWaitEvent(aux, c->ev_rev[buf ^ 1], 0));
      rs = recompute(s - 1);
      if (rs != LBM_OK) return rs;
    }
    CUDA_OK(c, cudaStreamWaitEvent(st, c->ev_rec[buf], 0));
    CUDA_OK(c, cudaGraphLaunch(find(1, buf, k, p), st));
    CUDA_OK(c, cudaEventRecord(c->ev_rev[buf], st));
    p ^= (int)(k & 1);
  }
  if (df0) {
    real* dst = on_device ? (real*)df0 : (real*)(w + A.lam_bc);
    CUDA_OK(c, adj_export(L, lam[p], (const real*)(w + A.Lrho), dst, st));
    if (!on_device) CUDA_OK(c, cudaMemcpyAsync(df0, dst, 9 * dn * y.sz, cudaMemcpyDeviceToHost, st));
  }
  std::vector<double> g(3 * c->cfg.n_cyl + 1);
  CUDA_OK(c, cudaMemcpyAsync(g.data(), w + A.grad, g.size() * 8, cudaMemcpyDeviceToHost, st));
  // the forward state as it was after lbm_forward_checkpointed
  CUDA_OK(c, cudaMemcpyAsync(L.dM_ring, w + A.ring, (size_t)(DM_RING + 1) * 8, cudaMemcpyDeviceToDevice, st));
  CUDA_OK(c, cudaMemcpyAsync(L.step_ctr, w + A.ctr, 8, cudaMemcpyDeviceToDevice, st));
  if (c->n_bnodes > 0)
    CUDA_OK(c, cudaMemcpyAsync(L.carry, w + A.carry, (size_t)c->n_bnodes * 8, cudaMemcpyDeviceToDevice, st));
  CUDA_OK(c, cudaStreamSynchronize(st));
  if (grad) std::memcpy(grad, g.data(), g.size() * 8);
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_adjoint_workspace_size(lbm_ctx* c, int64_t n_steps, int64_t every, size_t* bytes) {
  if (!c || !c->built || !bytes) return LBM_ESTATE;
  if (c->cfg.force_model != LBM_FORCE_CHEMPOT) return fail(c, LBM_EINVAL, "the reverse mode covers the chemical-potential force only");
  if (c->cfg.layout != LBM_LAYOUT_AB) return fail(c, LBM_EINVAL, "the reverse mode needs two population lattices");
  if (n_steps < 1 || every < 0) return fail(c, LBM_EINVAL, "n_steps must be positive and every non-negative");
  *bytes = make_adj_layout(c, n_steps, every).total;
  return LBM_OK;
}

lbm_status lbm_forward_checkpointed(lbm_ctx* c, int64_t n_steps, int64_t every, void* workspace, size_t bytes) {
  LBM_RANGE("lbm_forward_checkpointed");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (n_steps < 1 || every < 0) return fail(c, LBM_EINVAL, "n_steps must be positive and every non-negative");
  if (c->cfg.force_model != LBM_FORCE_CHEMPOT) return fail(c, LBM_EINVAL, "the reverse mode covers the chemical-potential force only");
  if (c->cfg.layout != LBM_LAYOUT_AB) return fail(c, LBM_EINVAL, "the reverse mode needs two population lattices");
  const AdjLayout A = make_adj_layout(c, n_steps, every);
  if (!workspace || ((uintptr_t)workspace) % ALIGN) return fail(c, LBM_EINVAL, "adjoint workspace must be 256-byte aligned");
  if (bytes < A.total) return fail(c, LBM_ENOMEM, "adjoint workspace of %zu bytes, %zu needed", bytes, A.total);
  c->tape = lbm_ctx::Tape{};
  c->tape.ws = (char*)workspace;
  c->tape.bytes = bytes;
  c->tape.n = A.n;
  c->tape.every = A.every;
  c->tape.nseg = A.nseg;
  lbm_status s = c->fp64 ? forward_checkpointed(c, c->Ld, A) : forward_checkpointed(c, c->Lf, A);
  if (s != LBM_OK) return s;
  c->tape.steps_end = c->steps;
  c->tape.cur_end = c->cur;
  c->tape.valid = true;
  return LBM_OK;
}

lbm_status lbm_objective(lbm_ctx* c, int32_t body, double* J, void* dJ_drho, int32_t on_device) {
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!J) return fail(c, LBM_EINVAL, "null output");
  if (body < 0 || body >= c->cfg.n_cyl) return fail(c, LBM_EINVAL, "body %d is not a cylinder", body);
  if (c->cfg.layout != LBM_LAYOUT_AB) return fail(c, LBM_EINVAL, "the reverse mode needs two population lattices");
  return c->fp64 ? objective(c, c->Ld, body, J, dJ_drho, on_device) : objective(c, c->Lf, body, J, dJ_drho, on_device);
}

lbm_status lbm_adjoint(lbm_ctx* c, const void* dJ_drho, const void* dJ_df, int32_t on_device, double* grad,
                       void* dJ_df0) {
  LBM_RANGE("lbm_adjoint");
  if (!c || !c->inited) return LBM_ESTATE;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!c->tape.valid || c->tape.steps_end != c->steps || c->tape.cur_end != c->cur)
    return fail(c, LBM_ESTATE, "no checkpointed forward pass ends at the current state");
  return c->fp64 ? adjoint(c, c->Ld, dJ_drho, dJ_df, on_device, grad, dJ_df0)
                 : adjoint(c, c->Lf, dJ_drho, dJ_df, on_device, grad, dJ_df0);
}

}  // extern "C"
