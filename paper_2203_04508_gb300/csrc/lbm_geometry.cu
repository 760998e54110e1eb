// Geometry set-up on the device: node classes, cut links with their fractions q, and the
// solid-layer lists of the wetting boundary (Sec. 2.3, Sec. 3.1).
//
// This translation unit is compiled with -fmad=false: q is evaluated in FP64 with every
// product and sum rounded separately, in a fixed order, so that the same inputs give the
// same bits on any IEEE-754 host:
//   dx = x - cx, dy = y - cy, A = |e_i|^2, B = 2 (dx e_x + dy e_y), C = (dx^2 + dy^2) - r^2,
//   q = (-B - sqrt(B^2 - 4 A C)) / (2 A)      (smaller root of |x1 + q e_i - c|^2 = r^2)
// and q = y1 - y_bottom or y_top - y1 for the flat walls.  A node is solid when
// dx^2 + dy^2 <= r^2 (nodes on the circle are solid) or y <= y_bottom or y >= y_top.
#include <climits>

#include "lbm_internal.h"

namespace lbmgb {

constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ int gwrap_x(const GeomParams& g, int x) { return x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x); }

// neighbour of (x, y) along e_i; false when it leaves a walled domain in y
__device__ __forceinline__ bool gnb(const GeomParams& g, int x, int y, int i, int* m) {
  int xx = gwrap_x(g, x + ex(i));
  int yy = y + ey(i);
  if (g.walls) {
    if (yy < 0 || yy >= g.ny) return false;
  } else {
    yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
  }
  *m = yy * g.pitch + xx;
  return true;
}

// global row of local row y (a slab's rows are a window of a larger lattice)
__device__ __forceinline__ int grow(const GeomParams& g, int y) {
  int r = y + g.y_off;
  if (g.ny_glob > 0) r = r < 0 ? r + g.ny_glob : (r >= g.ny_glob ? r - g.ny_glob : r);
  return r;
}

__device__ __forceinline__ bool inside_body(const GeomParams& g, int b, int x, int y) {
  if (b < g.n_cyl) {
    const double* c = g.cyl + 4 * b;
    double dx = (double)x - c[0];
    double dy = (double)grow(g, y) - c[1];
    double d2 = dx * dx + dy * dy;
    return d2 <= c[2] * c[2];
  }
  if (b == g.n_cyl) return (double)y <= g.y_bottom;
  return (double)y >= g.y_top;
}

__device__ __forceinline__ double q_body(const GeomParams& g, int b, int x, int y, int i) {
  if (b < g.n_cyl) {
    const double* c = g.cyl + 4 * b;
    double dx = (double)x - c[0];
    double dy = (double)grow(g, y) - c[1];
    double A = (double)(ex(i) * ex(i) + ey(i) * ey(i));
    double B = 2.0 * (dx * (double)ex(i) + dy * (double)ey(i));
    double C = (dx * dx + dy * dy) - c[2] * c[2];
    double disc = B * B - 4.0 * A * C;
    return (-B - sqrt(disc)) / (2.0 * A);
  }
  if (b == g.n_cyl) return (double)y - g.y_bottom;
  return g.y_top - (double)y;
}

// An FP32 screen of the disc test of inside_body, exact where it decides.  For node
// coordinates, centres and radii below 2^13 the FP32 d^2 lies within 134 of the exact one (the
// centre and the difference rounded once each, 2^-10 in all; the two squares and their sum),
// and the FP64 d^2 and r^2 within 1e-6 of theirs; so d2f > r^2 + 256 and d2f < r^2 - 256, with
// both bounds rounded to FP32 (within 4), give the FP64 test's answer.  Nodes in the ring
// between the bounds, and centres or radii out of range (bounds -inf, +inf), take the FP64
// test.  GB300's FP64 rate makes the plain test the cost of the classification.
constexpr int SCREEN_MAX = 32;
constexpr int SCREEN_COORD = 8192;

__device__ __forceinline__ float4 disc_screen(const double* c) {
  const bool ok = fabs(c[0]) < (double)SCREEN_COORD && fabs(c[1]) < (double)SCREEN_COORD && c[2] >= 0.0 &&
                  c[2] < (double)SCREEN_COORD;
  if (!ok) return make_float4(0.f, 0.f, __int_as_float((int)0xff800000), __int_as_float(0x7f800000));
  const double r2 = c[2] * c[2];
  return make_float4((float)c[0], (float)c[1], (float)(r2 - 256.0), (float)(r2 + 256.0));
}

// 1 inside, 0 outside, -1 undecided
__device__ __forceinline__ int screen_disc(float4 s, int x, int gy) {
  const float dx = (float)x - s.x, dy = (float)gy - s.y;
  const float d2 = dx * dx + dy * dy;
  return d2 > s.w ? 0 : (d2 < s.z ? 1 : -1);
}

// The flat walls' tests (double)y <= y_bottom and (double)y >= y_top for integer rows y in
// [0, 2^30): y <= floor(y_bottom) and y >= ceil(y_top), with NaN bounds never met.
__device__ __forceinline__ int wall_lo_row(double yb) {
  if (!(yb >= -1073741824.0)) return INT_MIN / 2;
  return yb >= 1073741824.0 ? 1073741824 : (int)floor(yb);
}
__device__ __forceinline__ int wall_hi_row(double yt) {
  if (!(yt <= 1073741824.0)) return INT_MAX / 2;
  return yt <= -1073741824.0 ? -1073741824 : (int)ceil(yt);
}

// grid (ceil(pitch / 256), up to GEOM_ROW_BLOCKS), 256 threads: one node of a row each, rows
// blockIdx.y, blockIdx.y + gridDim.y, ... (the per-block set-up is paid once for all of them)
constexpr int GEOM_ROW_BLOCKS = 512;
__global__ void __launch_bounds__(256) k_classify(GeomParams g, uint8_t* kind, int* body) {
  __shared__ float4 scr[SCREEN_MAX];
  __shared__ int wl, wh;
  const int ns = g.n_cyl < SCREEN_MAX ? g.n_cyl : SCREEN_MAX;
  if ((int)threadIdx.x < ns) scr[threadIdx.x] = disc_screen(g.cyl + 4 * threadIdx.x);
  if (threadIdx.x == 0) { wl = wall_lo_row(g.y_bottom); wh = wall_hi_row(g.y_top); }
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.pitch) return;
  const int rows = (int)(g.plane / g.pitch);
  for (int y = blockIdx.y; y < rows; y += gridDim.y) {
    const long long n = (long long)y * g.pitch + x;
    if (x >= g.nx) { kind[n] = KIND_PAD; body[n] = -1; continue; }
    const int gy = grow(g, y);
    const bool fast = x < SCREEN_COORD && gy >= 0 && gy < SCREEN_COORD;
    int bd = -1;
    for (int b = 0; b < g.n_cyl; ++b) {
      int in = fast && b < SCREEN_MAX ? screen_disc(scr[b], x, gy) : -1;
      if (in < 0) in = inside_body(g, b, x, y) ? 1 : 0;
      if (in) { bd = b; break; }
    }
    if (bd < 0 && g.walls) {
      if (y <= wl) bd = g.n_cyl;
      else if (y >= wh) bd = g.n_cyl + 1;
    }
    body[n] = bd;
    kind[n] = bd >= 0 ? KIND_DEEP : KIND_FLUID;
  }
}

// solid nodes with a neighbour of class `from` (and currently DEEP) become class `to`
// the same grid as k_classify
__global__ void __launch_bounds__(256) k_layer(GeomParams g, uint8_t* kind, uint8_t from, uint8_t to) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.pitch) return;
  const int rows = (int)(g.plane / g.pitch);
  for (int y = blockIdx.y; y < rows; y += gridDim.y) {
    const long long n = (long long)y * g.pitch + x;
    if (kind[n] != KIND_DEEP) continue;
    for (int i = 1; i < 9; ++i) {
      int m;
      if (gnb(g, x, y, i, &m) && kind[m] == from) { kind[n] = to; break; }
    }
  }
}

// ---- the four lists (cut links, boundary nodes, first and second solid layer) and the fluid
// count, compacted in node order: per block of LIST_NODES consecutive nodes (LIST_NPT
// consecutive nodes of one row a thread) the counts of each list are scanned in shared memory;
// one scan over the blocks' totals gives each block's offsets.
enum { LANE_LINKS = 0, LANE_BNODE, LANE_S1, LANE_S2, LANE_FLUID, N_LANES };
constexpr int LIST_BLOCK = 256, LIST_NPT = 8, LIST_NODES = LIST_BLOCK * LIST_NPT;

// Bit offsets of the five lanes in one packed 64-bit count: a block of LIST_NODES = 2048 nodes
// holds at most 8 x 2048 cut links (15 bits) and 2048 of each other lane (in fields of 12 bits),
// so a block scan of the packed counts never carries from one field into the next
// (bits 0, 15, 27, 39, 51).
__host__ __device__ constexpr int lane_shift(int l) { return l == 0 ? 0 : 3 + 12 * l; }

__device__ __forceinline__ int lane_of_packed(unsigned long long v, int l) {
  return (int)((v >> lane_shift(l)) & (l == 0 ? 0x7fffull : 0xfffull));
}

// packed counts of node (x, y) of class k: its cut links (a fluid node with a non-fluid
// neighbour), the boundary-node, layer flags and the fluid flag
__device__ __forceinline__ unsigned long long node_counts(const GeomParams& g, const uint8_t* kind, uint8_t k, int x,
                                                          int y) {
  if (k == KIND_FLUID) {
    int links = 0;
    for (int i = 1; i < 9; ++i) {
      int m;
      if (gnb(g, x, y, i, &m) && kind[m] != KIND_FLUID) ++links;
    }
    return ((unsigned long long)links << lane_shift(LANE_LINKS)) |
           ((unsigned long long)(links > 0) << lane_shift(LANE_BNODE)) | (1ull << lane_shift(LANE_FLUID));
  }
  if (k == KIND_SOLID1) return 1ull << lane_shift(LANE_S1);
  if (k == KIND_SOLID2) return 1ull << lane_shift(LANE_S2);
  return 0ull;
}

// The LIST_NPT nodes of thread threadIdx.x: its first node n0 (returned; >= plane for threads
// past the end), their row y and first column x0 (all in one row: the pitch is a multiple of 32
// and blocks start at multiples of LIST_NODES), their classes and packed counts.  The block's
// first node is divided by the pitch once, by thread 0.
__device__ __forceinline__ long long thread_counts(const GeomParams& g, const uint8_t* kind, int* x0, int* y,
                                                   uint8_t (&k)[LIST_NPT], unsigned long long (&c)[LIST_NPT]) {
  __shared__ int b0[2];
  const long long base = (long long)blockIdx.x * LIST_NODES;
  if (threadIdx.x == 0) {
    const long long r = base / g.pitch;
    b0[0] = (int)r;
    b0[1] = (int)(base - r * g.pitch);
  }
  __syncthreads();
  const unsigned t = (unsigned)b0[1] + LIST_NPT * threadIdx.x;
  *y = b0[0] + (int)(t / (unsigned)g.pitch);
  *x0 = (int)(t % (unsigned)g.pitch);
  const long long n0 = base + LIST_NPT * threadIdx.x;
  if (n0 >= g.plane) {
#pragma unroll
    for (int j = 0; j < LIST_NPT; ++j) { k[j] = KIND_PAD; c[j] = 0ull; }
    return n0;
  }
  const uint2 kk = *reinterpret_cast<const uint2*>(kind + n0);
#pragma unroll
  for (int j = 0; j < LIST_NPT; ++j) {
    k[j] = (uint8_t)(((j < 4 ? kk.x : kk.y) >> (8 * (j & 3))) & 0xffu);
    c[j] = node_counts(g, kind, k[j], *x0 + j, *y);
  }
  return n0;
}

// ---- block scans of int32 and packed 64-bit counts
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename T>
__device__ T block_excl_scan(T v, T* total) {
  __shared__ T ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    T s = lane < nw ? ws[lane] : T(0);
    s = warp_incl_scan(s);
    ws[lane] = s;
  }
  __syncthreads();
  T base = warp > 0 ? ws[warp - 1] : T(0);
  *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + inc - v;
}

// per block and lane the block's total, at sums[lane * nb + block]
__global__ void __launch_bounds__(LIST_BLOCK) k_count_blocks(GeomParams g, const uint8_t* kind, int* sums, int nb) {
  int x0, y;
  uint8_t k[LIST_NPT];
  unsigned long long c[LIST_NPT];
  (void)thread_counts(g, kind, &x0, &y, k, c);
  unsigned long long sum = 0ull, t;
#pragma unroll
  for (int j = 0; j < LIST_NPT; ++j) sum += c[j];
  (void)block_excl_scan(sum, &t);
  if (threadIdx.x < N_LANES) sums[threadIdx.x * nb + blockIdx.x] = lane_of_packed(t, threadIdx.x);
}

// one block per lane: exclusive scan of the lane's nb block totals in place, the lane's grand
// total to totals[lane]
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_lanes(int* sums, int nb, int* totals) {
  int* s = sums + (long long)blockIdx.x * nb;
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? s[i] : 0;
    int t;
    const int e = block_excl_scan(v, &t);
    if (i < nb) s[i] = e + carry;
    carry += t;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

cudaError_t geom_classify_and_count(const GeomParams& g, const GeomScratch& s, uint8_t* kind, cudaStream_t st) {
  const long long rows = g.plane / g.pitch;
  const dim3 grid((unsigned)((g.pitch + 255) / 256), (unsigned)(rows < GEOM_ROW_BLOCKS ? rows : GEOM_ROW_BLOCKS));
  k_classify<<<grid, 256, 0, st>>>(g, kind, s.body);
  k_layer<<<grid, 256, 0, st>>>(g, kind, KIND_FLUID, KIND_SOLID1);
  k_layer<<<grid, 256, 0, st>>>(g, kind, KIND_SOLID1, KIND_SOLID2);
  // totals: 0 links, 1 bnodes, 2 s1, 3 s2, 4 fluid
  const int nb = (int)((g.plane + LIST_NODES - 1) / LIST_NODES);
  k_count_blocks<<<nb, LIST_BLOCK, 0, st>>>(g, kind, s.block_sums, nb);
  k_scan_lanes<<<N_LANES, SCAN_BLOCK, 0, st>>>(s.block_sums, nb, s.totals);
  return cudaGetLastError();
}

// Each node's place in the lists: the boundary-node list (node, first link) and the two layer
// lists (node), and the boundary index of every boundary node in the plane bidx (read back for
// the first layer's neighbour table; other entries are never read).  The block offsets are the
// scanned totals k_scan_lanes left.
__global__ void __launch_bounds__(LIST_BLOCK) k_fill_nodes(GeomParams g, const uint8_t* kind, const int* offs, int nb,
                                                           GeomOut o, int* bidx) {
  int x0, y;
  uint8_t k[LIST_NPT];
  unsigned long long c[LIST_NPT];
  const long long n0 = thread_counts(g, kind, &x0, &y, k, c);
  unsigned long long sum = 0ull, t;
#pragma unroll
  for (int j = 0; j < LIST_NPT; ++j) sum += c[j];
  unsigned long long ex = block_excl_scan(sum, &t);
  int off[LANE_FLUID];
#pragma unroll
  for (int l = 0; l < LANE_FLUID; ++l) off[l] = offs[l * nb + blockIdx.x];
#pragma unroll
  for (int j = 0; j < LIST_NPT; ++j) {
    const long long n = n0 + j;
    if (lane_of_packed(c[j], LANE_BNODE)) {
      const int e = lane_of_packed(ex, LANE_BNODE) + off[LANE_BNODE];
      o.bnode[e] = (int)n;
      o.bstart[e] = lane_of_packed(ex, LANE_LINKS) + off[LANE_LINKS];
      bidx[n] = e;
    }
    if (lane_of_packed(c[j], LANE_S1)) o.s1node[lane_of_packed(ex, LANE_S1) + off[LANE_S1]] = (int)n;
    if (lane_of_packed(c[j], LANE_S2)) o.s2node[lane_of_packed(ex, LANE_S2) + off[LANE_S2]] = (int)n;
    ex += c[j];
  }
}

// The links of boundary node b, from its first link on, sorted by direction: direction, q (the
// nearest body's where a solid neighbour lies inside several), and whether x2 = x1 - e_i is fluid.
template <typename real>
__global__ void k_fill_links(GeomParams g, const uint8_t* kind, int n_bnodes, GeomOut o) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bnodes) return;
  const int n = o.bnode[b];
  const int x = n % g.pitch, y = n / g.pitch;
  int l = o.bstart[b];
  const int nbodies = g.n_cyl + (g.walls ? 2 : 0);
  for (int i = 1; i < 9; ++i) {
    int m;
    if (!gnb(g, x, y, i, &m) || kind[m] == KIND_FLUID) continue;
    int xs = m % g.pitch, ys = m / g.pitch;
    bool have = false;
    double qb = 0.0;
    for (int bd = 0; bd < nbodies; ++bd) {
      if (!inside_body(g, bd, xs, ys)) continue;
      double q = q_body(g, bd, x, y, i);
      if (!have || q < qb) { qb = q; have = true; }
    }
    int m2 = 0;
    bool ok2 = gnb(g, x, y, opp(i), &m2);
    o.ldir[l] = (uint8_t)i;
    o.lq64[l] = qb;
    ((real*)o.lq)[l] = (real)qb;
    o.lx2f[l] = (ok2 && kind[m2] == KIND_FLUID) ? 1 : 0;
    ++l;
  }
}

// Entry j of a solid-layer list (node[j] of class cls): the mask of its neighbours of class
// `from`, 1 / sum of their weights, and (first layer) for each contributing neighbour -- all of
// them boundary-fluid nodes -- its index in the boundary-node list, nb[8 j + i - 1], -1 where
// bit i-1 of the mask is clear
template <typename real>
__global__ void k_fill_layer(GeomParams g, const uint8_t* kind, int count, uint8_t from, const int* node,
                             uint8_t* mask, real* winv, const int* bidx, int* nb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const int n = node[j];
  const int x = n % g.pitch, y = n / g.pitch;
  unsigned msk = 0;
  double wsum = 0.0;
  for (int i = 1; i < 9; ++i) {
    int m;
    if (gnb(g, x, y, i, &m) && kind[m] == from) { msk |= 1u << (i - 1); wsum += wgt(i); }
  }
  mask[j] = (uint8_t)msk;
  winv[j] = (real)(1.0 / wsum);
  if (nb) {
    for (int i = 1; i < 9; ++i) {
      int m;
      nb[8 * j + i - 1] = (msk & (1u << (i - 1))) && gnb(g, x, y, i, &m) ? bidx[m] : -1;
    }
  }
}

// chemical potential plane (shifted by k^2 mu_sat): 0 at fluid and deep solid nodes, the
// wall offset dmu of the node's body at the two solid layers (Sec. 2.3)
template <typename real>
__global__ void k_wall_mu(GeomParams g, const uint8_t* kind, const int* body, real* mu) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.plane) return;
  uint8_t k = kind[n];
  real v = real(0);
  if (k == KIND_SOLID1 || k == KIND_SOLID2) {
    int b = body[n];
    v = (real)(b < g.n_cyl ? g.cyl[4 * b + 3] : g.dmu_walls);
  }
  mu[n] = v;
}

template <typename real>
static cudaError_t fill_typed(const GeomParams& g, const GeomScratch& s, const GeomOut& o, cudaStream_t st) {
  const unsigned gn = (unsigned)((g.plane + 255) / 256);
  const int nb = (int)((g.plane + LIST_NODES - 1) / LIST_NODES);
  // the block offsets geom_classify_and_count left in block_sums; the boundary index of each
  // boundary node into the scratch plane `off`
  int* bidx = s.off;
  k_fill_nodes<<<nb, LIST_BLOCK, 0, st>>>(g, o.kind, s.block_sums, nb, o, bidx);
  if (o.n_bnodes > 0) k_fill_links<real><<<(o.n_bnodes + 255) / 256, 256, 0, st>>>(g, o.kind, o.n_bnodes, o);
  if (o.n_s1 > 0)
    k_fill_layer<real><<<(o.n_s1 + 255) / 256, 256, 0, st>>>(g, o.kind, o.n_s1, KIND_FLUID, o.s1node, o.s1mask,
                                                             (real*)o.s1winv, bidx, o.s1nb);
  if (o.n_s2 > 0)
    k_fill_layer<real><<<(o.n_s2 + 255) / 256, 256, 0, st>>>(g, o.kind, o.n_s2, KIND_SOLID1, o.s2node, o.s2mask,
                                                             (real*)o.s2winv, nullptr, nullptr);
  k_wall_mu<real><<<gn, 256, 0, st>>>(g, o.kind, s.body, (real*)o.mu);
  return cudaGetLastError();
}

cudaError_t geom_fill(const GeomParams& g, const GeomScratch& s, const GeomOut& o, double, cudaStream_t st) {
  return o.fp64 ? fill_typed<double>(g, s, o, st) : fill_typed<float>(g, s, o, st);
}

}  // namespace lbmgb
