// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda.h>            // CUtensorMap (the type; the encoder is taken from the CUDA driver at run time)
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>   // header-only; a no-op unless a profiler attaches

#include "lbm_device.cuh"

namespace lbmgb {

// A named NVTX range around a host call, so that a timeline profiler shows the library's entry
// points (set-up, stepping, read-outs, checkpoints) over the kernels they launch.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define LBM_RANGE(name) ::lbmgb::NvtxRange lbm_nvtx_range_(name)

inline unsigned mass_blocks() { return 152 * 4; }

// ---- step kernels (lbm_step.cu)
template <typename real> cudaError_t launch_step(const Lattice<real>& L, int cur, cudaStream_t s);
template <typename real> int launches_per_step(const Lattice<real>& L);
template <typename real> cudaError_t launch_phase(const Lattice<real>& L, int cur, int phase, cudaStream_t s);
// the phases of a step whose collide kernel forms the next density (column sweeps), and whether
// the step from lattice cur runs that way
template <typename real>
cudaError_t launch_phase_sweep(const Lattice<real>& Lt, const Lattice<real>& Ln, int cur, int phase, cudaStream_t s);
template <typename real> bool step_sweeps(const Lattice<real>& L, int cur);
template <typename real> cudaError_t launch_macro(const Lattice<real>& L, int cur, cudaStream_t s);
// step t with its boundary phase and the next state's solid layers overlapping the density
// pass of step t+1 on stream s2 (Lt: rho = fluid and solid-layer densities of lattice cur,
// rho_b set; Ln: rho = the plane receiving lattice cur^1's).  Starts at the chemical potential.
template <typename real>
cudaError_t launch_step_overlap(const Lattice<real>& Lt, const Lattice<real>& Ln, int cur, cudaStream_t s,
                                cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join);
template <typename real> int launches_per_step_overlap(const Lattice<real>& L);
// one double into page-locked host memory (its device address dst), in stream order
cudaError_t launch_copy8(const double* src, double* dst, cudaStream_t s);
template <typename real> cudaError_t launch_fields(const Lattice<real>& L, int cur, real* r, real* vx, real* vy, cudaStream_t s);
// populations i0 <= i < i1 of the current state, population i into dense plane i - i0 of out
template <typename real>
cudaError_t launch_populations(const Lattice<real>& L, int cur, real* out, int i0, int i1, cudaStream_t s);
template <typename real>
cudaError_t launch_column(const Lattice<real>& L, int cur, int x, int y0, int n, double* out, cudaStream_t s);
template <typename real>
cudaError_t launch_max_speed(const Lattice<real>& L, int cur, unsigned long long* out, cudaStream_t s);
template <typename real>
cudaError_t launch_set_populations(const Lattice<real>& L, int cur, const real* in, int i0, int i1, cudaStream_t s);
template <typename real> cudaError_t launch_mass(const Lattice<real>& L, int cur, cudaStream_t s);
template <typename real> cudaError_t launch_init(const Lattice<real>& L, const double* drops, int n_drop, double W,
                                                 double rho_g, double rho_l, cudaStream_t s);

// TMA descriptors of one FP32 lattice for the pipelined collide kernel (host side; a launch
// copies the ones it needs into the kernel's parameters).
struct CollideTma {
  CUtensorMap f[2];             // the two population lattices as (x, y, plane), box 32 x 8 x 9
  CUtensorMap rho[2];           // the two density planes, box 40 x 12 (tile plus halo)
  CUtensorMap mu[2];            // the chemical-potential plane (and the second psi plane of the
                                // pseudopotential force, which alternates like the density), box 40 x 12
  const void* f_ptr[2];         // the planes the descriptors were made for: a lattice
  const void* rho_ptr[2];       // descriptor pointing elsewhere runs the plain kernel
  const void* mu_ptr[2];
  CUtensorMap f_pull;           // one lattice in AA order: its populations, box 40 x 10 x 9 from
                                // (x0 - 4, y0 - 1), for the second step's shifted rows
  bool pull_ok;                 // f_pull was encoded
  int blocks[2];                // persistent grid of the chemical-potential / psi variant
  int blocks_pull[2];           // ... of the AA order's second step
  int blocks_inplace[2];        // ... of its first step
  int sweep_blocks;             // blocks of the column-sweep variant that fit on the device at once
  float* edge;                  // its edge buffer (null: the sweep does not run)
};
// Encodes the descriptors for L (whose planes must not move afterwards) and sizes the grids;
// false, with a message, when the CUDA driver cannot.
bool collide_tma_setup(CollideTma* T, const Lattice<float>& L, const void* rho0, const void* rho1, const void* mu1,
                       void* edge, char* err);

// ---- halo messages of a y-slab (lbm_slab.cu)
constexpr int SLAB_PLANES = 11;   // nine populations, density, psi'(rho) - mu_sat or psi
struct SlabMsgLayout {
  long long cap;                  // carries a message can hold (H * nx)
  size_t carry, key, planes;      // byte offsets
  long long plane_elems;          // H * pitch
  size_t total;
};
SlabMsgLayout slab_msg_layout(int nrows, int pitch, int nx, int sz);
template <typename real>
cudaError_t launch_slab_pack(const Lattice<real>& L, int cur, real* rho, real* aux, int row0, int nrows, int b0,
                             int b1, void* msg, cudaStream_t s);
template <typename real>
cudaError_t launch_slab_unpack(const Lattice<real>& L, int cur, real* rho, real* aux, int row0, int nrows, int b0,
                               int b1, const void* msg, cudaStream_t s);

// ---- geometry (lbm_geometry.cu, compiled without FMA contraction)
struct GeomParams {
  int nx, ny, pitch, walls;
  long long plane;
  double y_bottom, y_top;
  int n_cyl;
  const double* cyl;          // device: n_cyl x {cx, cy, r, dmu}
  double dmu_walls;
  // y-slab: cylinders are tested at global row y + y_off (mod ny_glob when ny_glob > 0); the
  // flat walls stay in local rows.  A whole lattice has 0, 0.
  int y_off, ny_glob;
};

struct GeomScratch {
  int* body;                  // plane (kept: the body of every solid node)
  int* cnt;                   // plane
  int* off;                   // plane
  int* block_sums;            // 5 x (ceil(plane / 1024) + 1): per list and node block (2048 nodes)
  int* totals;                // 8 ints on the device
};

struct GeomOut {
  uint8_t* kind;
  int* bnode; int* bstart; uint8_t* ldir; double* lq64; uint8_t* lx2f;
  int* s1node; uint8_t* s1mask; int* s2node; uint8_t* s2mask;
  int* s1nb;                                // 8 per first-layer entry: neighbours' boundary index
  void* lq;   void* s1winv; void* s2winv;   // precision-typed
  void* mu;                                 // precision-typed plane
  int fp64;
  int n_bnodes, n_s1, n_s2;                 // list lengths (from the counts)
};

// Classification, layers and counts.  Leaves totals = {n_links, n_bnodes, n_s1, n_s2, n_fluid}
// on the device (and each node block's list offsets in block_sums) for the host to check
// capacities.
cudaError_t geom_classify_and_count(const GeomParams& g, const GeomScratch& s, uint8_t* kind, cudaStream_t st);
// Fills the link CSR, the layer lists and the constant wall chemical potential.
cudaError_t geom_fill(const GeomParams& g, const GeomScratch& s, const GeomOut& o, double k2_mu_sat_unused,
                      cudaStream_t st);

// ---- batched persistent step (lbm_batch.cu)
struct BatchDev {
  int n_inst;
  const void* lat;              // device array of n_inst Lattice<real> descriptors
  int groups;                   // 1: all instances in lockstep; 2: group 1 runs SKEW phases behind
  const uint8_t* inst_group;    // group of each instance
  // work lists, group 0's items first: group g's are [x_start[g], x_start[g+1])
  int tile_log2w;               // node tiles: width 2^tile_log2w, height 256 / 2^tile_log2w
  int tile_start[3], s1_start[3], s2_start[3], bc_start[3];
  const int2* node_tiles;       // (instance, tile), row-major over each instance's tiles
  const int2* s1_items;         // (instance, first entry) of 256 list entries
  const int2* s2_items;
  const int2* bc_items;
  const int2* inst_bc;          // bc items of instance k: [inst_bc[k].x, inst_bc[k].y)
  double* bc_partials;          // one compensation sum per bc item
  unsigned int* bar;            // grid barrier: arrivals, completed barriers
  unsigned long long* work;     // BATCH_WORK_COUNTERS work counters: items handed out in tick tau
                                // to group g at work[2 (tau % 3) + g] (zeroed before the launch)
  int* err;                     // set when a barrier wait gave up
  long long spin_limit;         // polls before a barrier wait gives up
};
int batch_block_size();
constexpr int BATCH_WORK_COUNTERS = 6;
// a second-solid-layer item (instance, first entry | BATCH_BMOM_ITEM) that saves the moments of
// 256 boundary nodes of a lattice in AA order instead
constexpr int BATCH_BMOM_ITEM = 1 << 30;
// node tiles of width 2^log2w (and height 256 / 2^log2w) of one instance; the shapes a batch
// may use are log2w = BATCH_TILE_LOG2W_MIN .. BATCH_TILE_LOG2W_MAX (16x16 .. 256x1)
constexpr int BATCH_TILE_LOG2W_MIN = 4, BATCH_TILE_LOG2W_MAX = 8, BATCH_TILE_LOG2W_DEFAULT = 5;
long long batch_node_tiles(int nx, int ny, int log2w);
int batch_grid_size(int fp64);
cudaError_t launch_batch(const BatchDev& B, int fp64, int grid, int n_steps, int cur0, cudaStream_t s);

// ---- reverse mode of the step (lbm_adjoint.cu)
// Precision-typed planes (pitch * ny elements each) of one reverse step.
struct AdjBuffers {
  const void* lam_in;   // 9 planes: dJ/df^{t+1}
  void* lam_out;        // 9 planes: dJ/df^t
  void* lam_bc;         // 9 planes: boundary contributions to dJ/d(post-collision f), zero between steps
  void* lrj;            // 3 planes: dJ/d(delta rho, jx, jy) of the link rule at boundary nodes
  void* lamF;           // 2 planes: dJ/dF (zero off the fluid)
  void* Lmu;            // dJ/dmu
  void* Lrho;           // dJ/drho (the density plane); between steps the density share of lambda
  const uint8_t* bct;   // per node: bit 0 lam_bc may be non-zero, bit 1 boundary node
  double* grad;         // dJ/d dmu per cylinder, dJ/d dmu of the walls, dJ/d(cx, cy) per cylinder
  int n_cyl;
};
// blocks of the objective's reduction over a plane of `plane` nodes (at most one per 256
// nodes): it leaves 4 partial sums per block in `red`
unsigned objective_blocks(long long plane);
template <typename real> cudaError_t adj_flags(const Lattice<real>& L, uint8_t* bct, cudaStream_t s);
template <typename real>
cudaError_t objective_sums(const Lattice<real>& L, int cur, int body, uint8_t* touch, double* red, double rg,
                           double rl, cudaStream_t s);
template <typename real>
cudaError_t objective_seed(const Lattice<real>& L, const uint8_t* touch, double y_cm, double S, double wcoef,
                           real* out, cudaStream_t s);
template <typename real>
cudaError_t adj_seed(const Lattice<real>& L, real* lam, const real* drho, const real* df, cudaStream_t s);
template <typename real>
cudaError_t adj_export(const Lattice<real>& L, const real* lam, const real* Lrho, real* out, cudaStream_t s);
template <typename real> cudaError_t adj_step(const Lattice<real>& L, const AdjBuffers& A, cudaStream_t s);

// ---- EOS on the host (lbm_eos.cpp)
struct EosSolution {
  double Tc, rho_c, T, alpha, rho_g, rho_l, mu_sat, p_sat;
};
// returns 0 on success, otherwise writes a message to err (256 bytes)
int eos_solve(int kind, double a, double b, double R, double Tr, double omega, EosSolution* out, char* err);
double eos_pressure(int kind, double a, double b, double RT, double aalpha, double rho);
double eos_mu(int kind, double a, double b, double RT, double aalpha, double rho);

}  // namespace lbmgb
