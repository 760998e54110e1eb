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

__global__ void k_classify(GeomParams g, uint8_t* kind, int* body) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.plane) return;
  int x = (int)(n % g.pitch), y = (int)(n / g.pitch);
  if (x >= g.nx) { kind[n] = KIND_PAD; body[n] = -1; return; }
  int nb = g.n_cyl + (g.walls ? 2 : 0);
  int bd = -1;
  for (int b = 0; b < nb; ++b)
    if (inside_body(g, b, x, y)) { bd = b; break; }
  body[n] = bd;
  kind[n] = bd >= 0 ? KIND_DEEP : KIND_FLUID;
}

// solid nodes with a neighbour of class `from` (and currently DEEP) become class `to`
__global__ void k_layer(GeomParams g, uint8_t* kind, uint8_t from, uint8_t to) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.plane) return;
  if (kind[n] != KIND_DEEP) return;
  int x = (int)(n % g.pitch), y = (int)(n / g.pitch);
  for (int i = 1; i < 9; ++i) {
    int m;
    if (gnb(g, x, y, i, &m) && kind[m] == from) { kind[n] = to; return; }
  }
}

// what = 0: cut links of a fluid node; 1: boundary-fluid node flag; 2: layer-1 flag;
// 3: layer-2 flag; 4: fluid flag
__global__ void k_count(GeomParams g, const uint8_t* kind, int* cnt, int what) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.plane) return;
  int x = (int)(n % g.pitch), y = (int)(n / g.pitch);
  uint8_t k = kind[n];
  int c = 0;
  if (what <= 1) {
    if (k == KIND_FLUID) {
      for (int i = 1; i < 9; ++i) {
        int m;
        if (gnb(g, x, y, i, &m) && kind[m] != KIND_FLUID) ++c;
      }
      if (what == 1) c = c > 0;
    }
  } else if (what == 2) {
    c = k == KIND_SOLID1;
  } else if (what == 3) {
    c = k == KIND_SOLID2;
  } else {
    c = k == KIND_FLUID;
  }
  cnt[n] = c;
}

// ---- deterministic exclusive scan of int32 counts (block scan, scan of block sums, add)
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ int block_excl_scan(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    int s = lane < nw ? ws[lane] : 0;
    s = warp_incl_scan(s);
    ws[lane] = s;
  }
  __syncthreads();
  int base = warp > 0 ? ws[warp - 1] : 0;
  *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + inc - v;
}

__global__ void k_scan_blocks(const int* in, int* out, int* block_sums, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int v = i < n ? in[i] : 0;
  int total;
  int e = block_excl_scan(v, &total);
  if (i < n) out[i] = e;
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// single block: exclusive scan of nb block sums in place; grand total to *total
__global__ void k_scan_sums(int* block_sums, int nb, int* total) {
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nb ? block_sums[i] : 0;
    int t;
    int e = block_excl_scan(v, &t);
    if (i < nb) block_sums[i] = e + carry;
    carry += t;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int* out, const int* block_sums, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += block_sums[blockIdx.x];
}

static cudaError_t excl_scan(const int* in, int* out, int* block_sums, int* total, long long n, cudaStream_t st) {
  unsigned nb = (unsigned)((n + SCAN_BLOCK - 1) / SCAN_BLOCK);
  k_scan_blocks<<<nb, SCAN_BLOCK, 0, st>>>(in, out, block_sums, n);
  k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(block_sums, (int)nb, total);
  k_scan_add<<<nb, SCAN_BLOCK, 0, st>>>(out, block_sums, n);
  return cudaGetLastError();
}

cudaError_t geom_classify_and_count(const GeomParams& g, const GeomScratch& s, uint8_t* kind, cudaStream_t st) {
  const unsigned gn = (unsigned)((g.plane + 255) / 256);
  k_classify<<<gn, 256, 0, st>>>(g, kind, s.body);
  k_layer<<<gn, 256, 0, st>>>(g, kind, KIND_FLUID, KIND_SOLID1);
  k_layer<<<gn, 256, 0, st>>>(g, kind, KIND_SOLID1, KIND_SOLID2);
  // totals: 0 links, 1 bnodes, 2 s1, 3 s2, 4 fluid
  for (int w = 0; w < 5; ++w) {
    k_count<<<gn, 256, 0, st>>>(g, kind, s.cnt, w);
    cudaError_t e = excl_scan(s.cnt, s.off, s.block_sums, s.totals + w, g.plane, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// link CSR: per boundary node its first link; links sorted by (node, direction)
template <typename real>
__global__ void k_fill_links(GeomParams g, const uint8_t* kind, const int* link_off, const int* bnode_off,
                             GeomOut o) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.plane) return;
  if (kind[n] != KIND_FLUID) return;
  int x = (int)(n % g.pitch), y = (int)(n / g.pitch);
  int base = link_off[n];
  int l = base;
  int nbodies = g.n_cyl + (g.walls ? 2 : 0);
  for (int i = 1; i < 9; ++i) {
    int m;
    if (!gnb(g, x, y, i, &m) || kind[m] == KIND_FLUID) continue;
    int xs = m % g.pitch, ys = m / g.pitch;
    bool have = false;
    double qb = 0.0;
    for (int b = 0; b < nbodies; ++b) {
      if (!inside_body(g, b, xs, ys)) continue;
      double q = q_body(g, b, x, y, i);
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
  if (l > base) {
    int b = bnode_off[n];
    o.bnode[b] = (int)n;
    o.bstart[b] = base;
  }
}

// bidx, nb (first layer only): for each contributing neighbour (all of them are boundary-fluid
// nodes) its index in the boundary-node list, nb[8 j + i - 1], -1 where bit i-1 of the mask is
// clear
template <typename real>
__global__ void k_fill_layer(GeomParams g, const uint8_t* kind, const int* off, uint8_t cls, uint8_t from,
                             int* node, uint8_t* mask, real* winv, const int* bidx, int* nb) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.plane) return;
  if (kind[n] != cls) return;
  int x = (int)(n % g.pitch), y = (int)(n / g.pitch);
  unsigned msk = 0;
  double wsum = 0.0;
  for (int i = 1; i < 9; ++i) {
    int m;
    if (gnb(g, x, y, i, &m) && kind[m] == from) { msk |= 1u << (i - 1); wsum += wgt(i); }
  }
  int j = off[n];
  node[j] = (int)n;
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
  double v = 0.0;
  if (k == KIND_SOLID1 || k == KIND_SOLID2) {
    int b = body[n];
    v = b < g.n_cyl ? g.cyl[4 * b + 3] : g.dmu_walls;
  }
  mu[n] = (real)v;
}

template <typename real>
static cudaError_t fill_typed(const GeomParams& g, const GeomScratch& s, const GeomOut& o, cudaStream_t st) {
  const unsigned gn = (unsigned)((g.plane + 255) / 256);
  // per-node link offsets (scratch `off`) and boundary-node offsets (scratch `cnt`, scanned
  // in place: each thread reads its element before any thread writes it)
  int* link_off = s.off;
  k_count<<<gn, 256, 0, st>>>(g, o.kind, s.cnt, 0);
  cudaError_t e = excl_scan(s.cnt, link_off, s.block_sums, s.totals + 5, g.plane, st);
  if (e != cudaSuccess) return e;
  k_count<<<gn, 256, 0, st>>>(g, o.kind, s.cnt, 1);
  e = excl_scan(s.cnt, s.cnt, s.block_sums, s.totals + 6, g.plane, st);
  if (e != cudaSuccess) return e;
  k_fill_links<real><<<gn, 256, 0, st>>>(g, o.kind, link_off, s.cnt, o);
  // the boundary-node index of every boundary node (the scan just used) outlives the link
  // offsets: keep it for the first layer's neighbour table
  int* bidx = s.off;
  e = cudaMemcpyAsync(bidx, s.cnt, (size_t)g.plane * sizeof(int), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  // layer 1 list
  k_count<<<gn, 256, 0, st>>>(g, o.kind, s.cnt, 2);
  e = excl_scan(s.cnt, s.cnt, s.block_sums, s.totals + 7, g.plane, st);
  if (e != cudaSuccess) return e;
  k_fill_layer<real><<<gn, 256, 0, st>>>(g, o.kind, s.cnt, KIND_SOLID1, KIND_FLUID, o.s1node, o.s1mask,
                                         (real*)o.s1winv, bidx, o.s1nb);
  // layer 2 list
  k_count<<<gn, 256, 0, st>>>(g, o.kind, s.cnt, 3);
  e = excl_scan(s.cnt, s.cnt, s.block_sums, s.totals + 7, g.plane, st);
  if (e != cudaSuccess) return e;
  k_fill_layer<real><<<gn, 256, 0, st>>>(g, o.kind, s.cnt, KIND_SOLID2, KIND_SOLID1, o.s2node, o.s2mask,
                                         (real*)o.s2winv, nullptr, nullptr);
  k_wall_mu<real><<<gn, 256, 0, st>>>(g, o.kind, s.body, (real*)o.mu);
  return cudaGetLastError();
}

cudaError_t geom_fill(const GeomParams& g, const GeomScratch& s, const GeomOut& o, double, cudaStream_t st) {
  return o.fp64 ? fill_typed<double>(g, s, o, st) : fill_typed<float>(g, s, o, st);
}

}  // namespace lbmgb
