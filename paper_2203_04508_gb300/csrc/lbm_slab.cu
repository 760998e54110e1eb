// Halo messages of the y-slab decomposition of one lattice (one context per slab).
//
// A slab context holds its own rows, an H-row halo on each side that has a neighbour, and two
// solid rows beyond each halo that terminate the local lattice.  A step reaches a node's state
// from at most seven rows away (streaming 1, the force stencil 2, the chemical-potential
// Laplacian 2, the two solid layers of Eq. 15 2), so after every step the H >= 7 halo rows are
// overwritten with the neighbour's own rows and the slab's own rows stay exactly those of the
// undivided lattice.  A message carries, for H consecutive rows of the current state:
//   - the nine population planes, the density plane (fluid nodes and the solid layers), and
//     the per-node EOS plane the next step starts from (psi'(rho) - mu_sat for the
//     chemical-potential force, psi for the pseudopotential force);
//   - the FP64 Eq. 18 carry of each boundary node in those rows, keyed by its position.
// Layout (bytes): [int64 count][8 pad][double carry[cap]][int32 key[cap]][pad to 16]
//                 [11 planes of H * pitch values], cap = H * nx.
#include "lbm_internal.h"

namespace lbmgb {

SlabMsgLayout slab_msg_layout(int nrows, int pitch, int nx, int sz) {
  auto up16 = [](size_t v) { return (v + 15) / 16 * 16; };
  SlabMsgLayout m{};
  m.cap = (long long)nrows * nx;
  m.carry = 16;
  m.key = up16(m.carry + (size_t)m.cap * 8);
  m.planes = up16(m.key + (size_t)m.cap * 4);
  m.plane_elems = (long long)nrows * pitch;
  m.total = up16(m.planes + (size_t)SLAB_PLANES * m.plane_elems * sz);
  return m;
}

namespace {

// rows [row0, row0 + nrows) of the 11 planes <-> the message
template <typename real, bool PACK>
__global__ void k_slab_planes(Lattice<real> L, int cur, real* rho, real* aux, int row0, int nrows,
                              real* __restrict__ msg_planes) {
  const long long per = (long long)nrows * L.pitch;
  const long long base = (long long)row0 * L.pitch;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < SLAB_PLANES * per;
       k += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(k / per);
    const long long e = k - (long long)p * per;
    real* plane = p < 9 ? L.f[cur] + (long long)p * L.plane : (p == 9 ? rho : aux);
    if (PACK) msg_planes[k] = plane[base + e];
    else plane[base + e] = msg_planes[k];
  }
}

// carries of boundary nodes [b0, b1) (the sender's rows) into the message, keyed by their
// position relative to the first row
template <typename real>
__global__ void k_slab_pack_carry(Lattice<real> L, int row0, int b0, int b1, long long* count, double* carry,
                                  int* key) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) *count = b1 - b0;
  if (k >= b1 - b0) return;
  carry[k] = L.carry[b0 + k];
  key[k] = L.bnode[b0 + k] - row0 * L.pitch;
}

// each of the receiver's boundary nodes [b0, b1) takes the carry of the sender's node at the
// same position (binary search in the sorted keys); a node the sender does not have (one that
// touches the solid rows terminating this slab) gets 0
template <typename real>
__global__ void k_slab_unpack_carry(Lattice<real> L, int row0, int b0, int b1, const long long* count,
                                    const double* carry, const int* key) {
  const int b = b0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= b1) return;
  const int want = L.bnode[b] - row0 * L.pitch;
  long long lo = 0, hi = *count;
  while (lo < hi) {
    const long long mid = (lo + hi) / 2;
    if (key[mid] < want) lo = mid + 1; else hi = mid;
  }
  L.carry[b] = (lo < *count && key[lo] == want) ? carry[lo] : 0.0;
}

unsigned grid_of(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152LL * 16) g = 152LL * 16;
  return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

template <typename real>
cudaError_t launch_slab_pack(const Lattice<real>& L, int cur, real* rho, real* aux, int row0, int nrows, int b0,
                             int b1, void* msg, cudaStream_t s) {
  const SlabMsgLayout m = slab_msg_layout(nrows, L.pitch, L.nx, (int)sizeof(real));
  char* p = static_cast<char*>(msg);
  k_slab_planes<real, true><<<grid_of(SLAB_PLANES * m.plane_elems, 256), 256, 0, s>>>(
      L, cur, rho, aux, row0, nrows, reinterpret_cast<real*>(p + m.planes));
  k_slab_pack_carry<real><<<grid_of((b1 - b0) > 0 ? b1 - b0 : 1, 256), 256, 0, s>>>(
      L, row0, b0, b1, reinterpret_cast<long long*>(p), reinterpret_cast<double*>(p + m.carry),
      reinterpret_cast<int*>(p + m.key));
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_slab_unpack(const Lattice<real>& L, int cur, real* rho, real* aux, int row0, int nrows, int b0,
                               int b1, const void* msg, cudaStream_t s) {
  const SlabMsgLayout m = slab_msg_layout(nrows, L.pitch, L.nx, (int)sizeof(real));
  const char* p = static_cast<const char*>(msg);
  k_slab_planes<real, false><<<grid_of(SLAB_PLANES * m.plane_elems, 256), 256, 0, s>>>(
      L, cur, rho, aux, row0, nrows, const_cast<real*>(reinterpret_cast<const real*>(p + m.planes)));
  if (b1 > b0)
    k_slab_unpack_carry<real><<<(unsigned)((b1 - b0 + 255) / 256), 256, 0, s>>>(
        L, row0, b0, b1, reinterpret_cast<const long long*>(p), reinterpret_cast<const double*>(p + m.carry),
        reinterpret_cast<const int*>(p + m.key));
  return cudaGetLastError();
}

template cudaError_t launch_slab_pack<float>(const Lattice<float>&, int, float*, float*, int, int, int, int, void*,
                                             cudaStream_t);
template cudaError_t launch_slab_pack<double>(const Lattice<double>&, int, double*, double*, int, int, int, int, void*,
                                              cudaStream_t);
template cudaError_t launch_slab_unpack<float>(const Lattice<float>&, int, float*, float*, int, int, int, int,
                                               const void*, cudaStream_t);
template cudaError_t launch_slab_unpack<double>(const Lattice<double>&, int, double*, double*, int, int, int, int,
                                                const void*, cudaStream_t);

}  // namespace lbmgb
