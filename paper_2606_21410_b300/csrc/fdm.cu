// Fast-diagonalization preconditioner M^{-1} for the collocation system
// (the paper solves without one; see the design notes).  M is the exact
// collocation operator with a constant conductivity kref and the same
// boundary rows.  Its block structure makes M^{-1} r exact:
//  - interior + single-face nodes: every face row of an interior a-line
//    couples only that line, so the two end values are eliminated per line
//    (u_b = G u_int + Binv g, the boundary elimination of Sec. 2.3.1), and
//    the reduced interior operator is the Kronecker sum kref (A_x + A_y + A_z)
//    of 1-D operators A_a = S_a Lambda_a S_a^{-1}; it is inverted by three
//    dense contractions with S^{-1}, a pointwise division by
//    kref (lx + ly + lz), and three contractions with S;
//  - edge / corner nodes: their boundary rows do not involve K; each is
//    solved on its owner axis' line (1x1 or 2x2) once the line interior is
//    known, edges before corners.
#include <algorithm>
#include <cstring>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "device.cuh"
#include "fdm.h"
#include "gemm.h"
#include "hostmath.h"
#include "umma.h"

namespace cheb {

// ---------------------------------------------------------------------------
// host set-up
// ---------------------------------------------------------------------------
template <typename T>
static int upload(T** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = (T)src[i];
  CHEB_CUDA(cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, tmp.size())));
  if (!tmp.empty()) CHEB_CUDA(cudaMemcpy(*dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice));
  return CHEB_OK;
}

static std::vector<double> transpose(const std::vector<double>& A, int r, int c) {
  std::vector<double> B((size_t)r * c);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) B[(size_t)j * r + i] = A[(size_t)i * c + j];
  return B;
}

// m x m matrix zero-padded to mp x mp
static std::vector<double> pad_square(const std::vector<double>& A, int m, int mp) {
  std::vector<double> B((size_t)mp * mp, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) B[(size_t)i * mp + j] = A[(size_t)i * m + j];
  return B;
}

static int pad4(int m) { return (m + 3) / 4 * 4; }

template <typename T>
static int upload_axis(FdmAxisDev<T>& d, const FdmAxisHost& h) {
  int st;
  const int m = h.m, mp = pad4(h.m);
  if ((st = upload(&d.S, pad_square(h.S, m, mp)))) return st;
  if ((st = upload(&d.Sinv, pad_square(h.Sinv, m, mp)))) return st;
  if ((st = upload(&d.ST, pad_square(transpose(h.S, m, m), m, mp)))) return st;
  if ((st = upload(&d.SinvT, pad_square(transpose(h.Sinv, m, m), m, mp)))) return st;
  std::vector<double> lam(mp, 0.0);
  for (int i = 0; i < m; ++i) lam[i] = h.lam[i];
  if ((st = upload(&d.lam, lam))) return st;
  if ((st = upload(&d.G, h.G))) return st;
  if ((st = upload(&d.Binv, h.Binv))) return st;
  if ((st = upload(&d.Lh, h.Lh))) return st;
  if ((st = upload(&d.Drow, h.Drow))) return st;
  return CHEB_OK;
}

// split-TF32 pair of the m x m matrix A, zero-padded to umma_n_tile(mp) x mp
static int upload_split(float** hi, float** lo, const std::vector<double>& A, int m, int mp) {
  const int rows = umma_n_tile(mp);
  std::vector<double> P((size_t)rows * mp, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) P[(size_t)i * mp + j] = A[(size_t)i * m + j];
  std::vector<float> h(P.size()), l(P.size());
  tf32_split_host(P.data(), P.size(), h.data(), l.data());
  CHEB_CUDA(cudaMalloc(hi, sizeof(float) * P.size()));
  CHEB_CUDA(cudaMalloc(lo, sizeof(float) * P.size()));
  CHEB_CUDA(cudaMemcpy(*hi, h.data(), sizeof(float) * P.size(), cudaMemcpyHostToDevice));
  CHEB_CUDA(cudaMemcpy(*lo, l.data(), sizeof(float) * P.size(), cudaMemcpyHostToDevice));
  return CHEB_OK;
}

template <typename T>
static void free_axis(FdmAxisDev<T>& d) {
  cudaFree(d.S); cudaFree(d.Sinv); cudaFree(d.ST); cudaFree(d.SinvT); cudaFree(d.lam);
  cudaFree(d.G); cudaFree(d.Binv); cudaFree(d.Lh); cudaFree(d.Drow);
  d = FdmAxisDev<T>();
}

// 1-D tables of axis a: end rows of the boundary conditions, elimination
// map, reduced interior operator and its eigen-decomposition.
static int build_axis_host(const cheb_plan_s* p, int a, FdmAxisHost& h) {
  const int n = p->n[a], N = n - 1, m = N - 1;
  h.n = n;
  h.m = m;
  const double scale = 2.0 / (p->hi[a] - p->lo[a]);
  std::vector<double> D = dense_deriv_matrix(N, scale);
  auto Dat = [&](int i, int j) { return D[(size_t)i * n + j]; };
  // end rows: index 0 is the hi face (2a+1, outward +), index N the lo face (2a, outward -)
  double B[4] = {0, 0, 0, 0};
  std::vector<double> Cm((size_t)2 * m, 0.0);
  if (p->bc[2 * a + 1] == CHEB_DIRICHLET) B[0] = 1.0;
  else {
    B[0] = Dat(0, 0); B[1] = Dat(0, N);
    for (int l = 0; l < m; ++l) Cm[l] = Dat(0, l + 1);
  }
  if (p->bc[2 * a] == CHEB_DIRICHLET) B[3] = 1.0;
  else {
    B[2] = -Dat(N, 0); B[3] = -Dat(N, N);
    for (int l = 0; l < m; ++l) Cm[m + l] = -Dat(N, l + 1);
  }
  const double det = B[0] * B[3] - B[1] * B[2];
  if (!(std::fabs(det) > 0)) { set_error("singular end-row block"); return CHEB_ERR_SINGULAR_BC; }
  h.Binv = {B[3] / det, -B[1] / det, -B[2] / det, B[0] / det};
  h.G.assign((size_t)2 * m, 0.0);
  for (int r = 0; r < 2; ++r)
    for (int l = 0; l < m; ++l)
      h.G[(size_t)r * m + l] = -(h.Binv[r * 2 + 0] * Cm[l] + h.Binv[r * 2 + 1] * Cm[m + l]);
  std::vector<double> D2 = matmul(D, D, n, n, n);
  // reduced operator A = -(D2_II + D2_IB G), lifting Lh = D2_IB Binv
  std::vector<double> Ared((size_t)m * m);
  h.Lh.assign((size_t)m * 2, 0.0);
  for (int i = 0; i < m; ++i) {
    const double b0 = D2[(size_t)(i + 1) * n + 0], bN = D2[(size_t)(i + 1) * n + N];
    for (int l = 0; l < m; ++l)
      Ared[(size_t)i * m + l] = -(D2[(size_t)(i + 1) * n + l + 1] + b0 * h.G[l] + bN * h.G[(size_t)m + l]);
    h.Lh[(size_t)i * 2 + 0] = b0 * h.Binv[0] + bN * h.Binv[2];
    h.Lh[(size_t)i * 2 + 1] = b0 * h.Binv[1] + bN * h.Binv[3];
  }
  if (!eig_real(Ared, m, h.lam, h.S)) {
    set_error("eigen-decomposition of the 1-D reduced operator failed");
    return CHEB_ERR_UNSUPPORTED;
  }
  h.Sinv = h.S;
  if (!invert(h.Sinv, m)) { set_error("singular eigenvector matrix"); return CHEB_ERR_UNSUPPORTED; }
  h.Drow.assign((size_t)2 * n, 0.0);
  for (int l = 0; l < n; ++l) {
    h.Drow[l] = Dat(0, l);
    h.Drow[(size_t)n + l] = Dat(N, l);
  }
  return CHEB_OK;
}

int fdm_setup(const cheb_plan_s* p, Fdm& f) {
  if (f.ready) return CHEB_OK;
  for (int a = 0; a < p->dim; ++a) {
    int st = build_axis_host(p, a, f.host[a]);
    if (st) return st;
    if ((st = upload_axis<double>(f.d64[a], f.host[a]))) return st;
    if ((st = upload_axis<float>(f.d32[a], f.host[a]))) return st;
  }
  for (int a = 0; a < 3; ++a) {
    f.m[a] = a < p->dim ? p->n[a] - 2 : 1;
    f.mp[a] = a < p->dim ? pad4(f.m[a]) : 1;
  }
  f.rot = false;
  if (p->dim >= 2 && !std::getenv("CHEB_FDM_NO_TCGEN05")) {
    const size_t ptot = (size_t)f.mp[0] * f.mp[1] * f.mp[2];
    bool ok = ptot < ((size_t)1 << 31);
    for (int a = 0; a < p->dim && ok; ++a) ok = umma_ok((int)(ptot / f.mp[a]), f.mp[a], f.mp[a]);
    if (ok) {
      for (int a = 0; a < p->dim; ++a) {
        const FdmAxisHost& h = f.host[a];
        const std::vector<double> mats[4] = {h.S, h.Sinv, transpose(h.S, h.m, h.m), transpose(h.Sinv, h.m, h.m)};
        for (int q = 0; q < 4; ++q) {
          int st = upload_split(&f.uw[a][2 * q], &f.uw[a][2 * q + 1], mats[q], h.m, f.mp[a]);
          if (st) return st;
        }
      }
      f.rot = true;
    }
  }
  f.ready = true;
  return CHEB_OK;
}

void fdm_free(Fdm& f) {
  for (int a = 0; a < 3; ++a) { free_axis(f.d64[a]); free_axis(f.d32[a]); }
  for (int a = 0; a < 3; ++a)
    for (int q = 0; q < 8; ++q) {
      cudaFree(f.uw[a][q]);
      f.uw[a][q] = nullptr;
    }
  f.rot = false;
  cudaFree(f.U64[0]); cudaFree(f.U64[1]); cudaFree(f.U32[0]); cudaFree(f.U32[1]);
  cudaFree(f.Y64); cudaFree(f.Y32);
  f.U64[0] = f.U64[1] = nullptr;
  f.U32[0] = f.U32[1] = nullptr;
  f.Y64 = nullptr;
  f.Y32 = nullptr;
  f.ready = false;
}

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------
template <typename T>
struct FdmK {
  const int* active;  // batched solves: skip while *active == 0 (null: always run)
  int m[3], mp[3], off[3];
  const T* Lh[3];
  const T* lam[3];
  const T* G[3];
  const T* Binv[3];
  const T* Drow[3];
};

// Grids have at most 257^3 points (axis sizes <= 257) and compact arrays
// at most 256^3 entries, so 32-bit index arithmetic is exact.
__device__ __forceinline__ uint32_t gidx3(const Geom& g, int i, int j, int k) {
  return ((uint32_t)k * (uint32_t)g.n[1] + (uint32_t)j) * (uint32_t)g.n[0] + (uint32_t)i;
}
// position of interior entry (ci, cj, ck) in the padded compact array
template <typename T>
__device__ __forceinline__ uint32_t cpos(const FdmK<T>& t, int ci, int cj, int ck) {
  return ((uint32_t)ck * (uint32_t)t.mp[1] + (uint32_t)cj) * (uint32_t)t.mp[0] + (uint32_t)ci;
}

// Element kernels run on a 3-D grid: x = (ci blocks of 128), y = cj, z = ck.
#define FDM_CELL_INDEX                                   \
  const int ci = blockIdx.x * blockDim.x + threadIdx.x; \
  const int cj = blockIdx.y, ck = blockIdx.z;           \
  if (ci >= t.m[0]) return;

// U (compact interior) = r_I + kref sum_a Lh_a (r at the two ends of the a-line).
// Grid (ceil(m_x / 128), m_y, ceil(m_z / kLiftK)): each thread takes kLiftK
// consecutive z entries of one (x, y) column (independent loads in flight;
// the z-end values of the column are read once).
constexpr int kLiftK = 8;
// (block coordinates explicit: the kernel below and the batched lift share it)
template <typename T>
__device__ __forceinline__ void fdm_lift_body(const Geom& g, const FdmK<T>& t, T kref, const T* __restrict__ r,
                                              T* __restrict__ U, int bx, int by, int bz) {
  if (t.active && *t.active == 0) return;  // converged batch instance
  const int ci = bx * blockDim.x + threadIdx.x, cj = by;
  if (ci >= t.m[0]) return;
  const int i = ci + t.off[0], j = cj + t.off[1];
  const int s1 = g.n[0], s2 = g.n[0] * g.n[1];
  const T lx0 = kref * t.Lh[0][2 * ci], lxN = kref * t.Lh[0][2 * ci + 1];
  const T ly0 = g.dim > 1 ? kref * t.Lh[1][2 * cj] : T(0), lyN = g.dim > 1 ? kref * t.Lh[1][2 * cj + 1] : T(0);
  T rz0 = 0, rzN = 0;
  if (g.dim > 2) {
    rz0 = r[j * s1 + i];
    rzN = r[(g.n[2] - 1) * s2 + j * s1 + i];
  }
  const int ck0 = bz * kLiftK, ck1 = min(ck0 + kLiftK, t.m[2]);
#pragma unroll 4
  for (int ck = ck0; ck < ck1; ++ck) {
    const int k = ck + t.off[2];
    const int p = k * s2 + j * s1 + i;
    T v = r[p] + lx0 * r[p - i] + lxN * r[p - i + g.n[0] - 1];
    if (g.dim > 1) v += ly0 * r[p - j * s1] + lyN * r[p + (g.n[1] - 1 - j) * s1];
    if (g.dim > 2) v += kref * (t.Lh[2][2 * ck] * rz0 + t.Lh[2][2 * ck + 1] * rzN);
    U[cpos(t, ci, cj, ck)] = v;
  }
}

template <typename T>
__global__ void fdm_lift_kernel(Geom g, FdmK<T> t, T kref, const T* __restrict__ r, T* __restrict__ U) {
  fdm_lift_body(g, t, kref, r, U, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T>
__global__ void fdm_scale_kernel(FdmK<T> t, int dim, T kref, T* __restrict__ U) {
  if (t.active && *t.active == 0) return;  // converged batch instance
  FDM_CELL_INDEX
  T l = t.lam[0][ci];
  if (dim > 1) l += t.lam[1][cj];
  if (dim > 2) l += t.lam[2][ck];
  const size_t q = cpos(t, ci, cj, ck);
  U[q] = U[q] / (kref * l);
}

template <typename T>
__global__ void fdm_scatter_kernel(Geom g, FdmK<T> t, const T* __restrict__ U, T* __restrict__ x) {
  if (t.active && *t.active == 0) return;  // converged batch instance
  FDM_CELL_INDEX
  x[gidx3(g, ci + t.off[0], cj + t.off[1], ck + t.off[2])] = U[cpos(t, ci, cj, ck)];
}

// Where the face step reads the interior values: src[off + ci + cj s1 + ck s2]
// (the compact array, or the interior of the full grid).
template <typename T>
struct FdmSrc {
  const T* p;
  long long off, s1, s2;
};

// End values of every interior x-line, [x0; xN] = G u_int(line) + Binv [r0; rN]:
// one warp per line (the line is contiguous); each lane keeps its eight
// entries of G (m <= 255 < 8 * 32) in registers for all its lines, loads its
// eight line values at once and the warp combines with shuffles.
template <typename T>
__device__ __forceinline__ void fdm_faces_x_body(const Geom& g, const FdmK<T>& t, const FdmSrc<T>& u,
                                                 const T* __restrict__ r, T* __restrict__ x, int blk,
                                                 int nblk) {
  if (t.active && *t.active == 0) return;  // converged batch instance
  const int ma = t.m[0];
  const int lines = t.m[1] * t.m[2];
  const int lane = threadIdx.x & 31;
  T g0[8], gN[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int l = lane + 32 * q;
    g0[q] = l < ma ? t.G[0][l] : T(0);
    gN[q] = l < ma ? t.G[0][ma + l] : T(0);
  }
  const T* Bi = t.Binv[0];
  const int nw = (nblk * blockDim.x) >> 5;
  for (int L = (blk * blockDim.x + threadIdx.x) >> 5; L < lines; L += nw) {
    const int cj = L % t.m[1], ck = L / t.m[1];
    const T* line = u.p + u.off + cj * u.s1 + ck * u.s2;
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int l = lane + 32 * q;
      v[q] = l < ma ? line[l] : T(0);
    }
    T s0 = 0, sN = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      s0 += g0[q] * v[q];
      sN += gN[q] * v[q];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      s0 += __shfl_down_sync(0xffffffffu, s0, d);
      sN += __shfl_down_sync(0xffffffffu, sN, d);
    }
    if (lane == 0) {
      const int j = cj + t.off[1], k = ck + t.off[2];
      const uint32_t p0 = gidx3(g, 0, j, k), pN = p0 + g.n[0] - 1;
      const T r0 = r[p0], rN = r[pN];
      x[p0] = s0 + Bi[0] * r0 + Bi[1] * rN;
      x[pN] = sN + Bi[2] * r0 + Bi[3] * rN;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) fdm_faces_x_kernel(Geom g, FdmK<T> t, FdmSrc<T> u,
                                                          const T* __restrict__ r, T* __restrict__ x) {
  fdm_faces_x_body(g, t, u, r, x, blockIdx.x, gridDim.x);
}

// Same for the y (a = 1) or z (a = 2) lines: a 32 x 8 block takes 32
// x-adjacent lines (coalesced reads), its 8 rows split the line and reduce
// through shared memory.  Grid: (ceil(m_x / 32), m_other).
template <typename T>
__device__ __forceinline__ void fdm_faces_yz_body(const Geom& g, const FdmK<T>& t, int a, const FdmSrc<T>& u,
                                                  const T* __restrict__ r, T* __restrict__ x, int bx,
                                                  int by) {
  if (t.active && *t.active == 0) return;  // converged batch instance
  __shared__ T red[2][8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int ci = bx * 32 + tx, co = by;
  const int ma = t.m[a];
  const long long sl = a == 1 ? u.s1 : u.s2, so = a == 1 ? u.s2 : u.s1;
  const T* G0 = t.G[a];
  const T* GN = t.G[a] + ma;
  T s0 = 0, sN = 0;
  if (ci < t.m[0]) {
    const T* line = u.p + u.off + ci + co * so;
#pragma unroll 4
    for (int l = ty; l < ma; l += 8) {
      const T v = line[l * sl];
      s0 += G0[l] * v;
      sN += GN[l] * v;
    }
  }
  red[0][ty][tx] = s0;
  red[1][ty][tx] = sN;
  __syncthreads();
  if (ty == 0 && ci < t.m[0]) {
    for (int q = 1; q < 8; ++q) {
      s0 += red[0][q][tx];
      sN += red[1][q][tx];
    }
    int e[3] = {ci + t.off[0], 0, 0};
    if (a == 1) e[2] = co + t.off[2];
    else e[1] = co + t.off[1];
    e[a] = 0;
    const size_t p0 = gidx3(g, e[0], e[1], e[2]);
    e[a] = g.n[a] - 1;
    const size_t pN = gidx3(g, e[0], e[1], e[2]);
    const T* Bi = t.Binv[a];
    const T r0 = r[p0], rN = r[pN];
    x[p0] = s0 + Bi[0] * r0 + Bi[1] * rN;
    x[pN] = sN + Bi[2] * r0 + Bi[3] * rN;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) fdm_faces_yz_kernel(Geom g, FdmK<T> t, int a, FdmSrc<T> u,
                                                           const T* __restrict__ r, T* __restrict__ x) {
  fdm_faces_yz_body(g, t, a, u, r, x, blockIdx.x, blockIdx.y);
}

// Boundary-row solve on a-lines that lie in one face (kind 1: the third
// index interior) or in two faces (kind 2), one warp per line.  End nodes
// owned by a Neumann face of axis a are solved from their rows
// s (D x)_e = r_e with the line interior known; Dirichlet-owned ends copy r;
// other ends belong to another axis' line and are left alone.  An a-line
// may read an end owned by a lower axis (never a higher one: at a shared
// end the lower axis wins among Neumann faces), so the axes run in
// increasing order, one launch each.
template <typename T>
__device__ __forceinline__ void fdm_bline_body(const Geom& g, const FdmK<T>& t, int a, int kind,
                                               const T* __restrict__ r, T* __restrict__ x, int blk, int nblk) {
  if (t.active && *t.active == 0) return;  // converged batch instance
  const int nb_axes = g.dim - 1;  // other active axes
  int others[2], no = 0;
  for (int q = 0; q < g.dim; ++q)
    if (q != a) others[no++] = q;
  // enumerate lines
  int total;
  if (kind == 1) {
    // (which other axis is on its face, side, interior index of the remaining axis)
    const int rem = (nb_axes == 2) ? 1 : 0;
    int cnt = 0;
    for (int q = 0; q < nb_axes; ++q) {
      const int cax = rem ? others[1 - q] : -1;
      cnt += 2 * (cax >= 0 ? g.n[cax] - 2 : 1);
    }
    total = cnt;
  } else {
    total = (nb_axes == 2) ? 4 : 0;
  }
  const int n = g.n[a], N = n - 1;
  const T* D0 = t.Drow[a];
  const T* DN = t.Drow[a] + n;
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int L = blk * wpb + (threadIdx.x >> 5); L < total; L += nblk * wpb) {
    int idx[3] = {0, 0, 0};
    if (kind == 1) {
      int rest = L, q = 0;
      for (; q < nb_axes; ++q) {
        const int cax = (nb_axes == 2) ? others[1 - q] : -1;
        const int span = 2 * (cax >= 0 ? g.n[cax] - 2 : 1);
        if (rest < span) break;
        rest -= span;
      }
      const int bax = others[q];
      const int cax = (nb_axes == 2) ? others[1 - q] : -1;
      const int side = rest & 1, tt = rest >> 1;
      idx[bax] = side ? 0 : g.n[bax] - 1;  // side 1 (hi) is index 0
      if (cax >= 0) idx[cax] = 1 + tt;
    } else {
      idx[others[0]] = (L & 1) ? 0 : g.n[others[0]] - 1;
      idx[others[1]] = (L & 2) ? 0 : g.n[others[1]] - 1;
    }
    int e[3] = {idx[0], idx[1], idx[2]};
    e[a] = 0;
    const size_t p0 = gidx3(g, e[0], e[1], e[2]);
    const int o0 = owner_face(g, e[0], e[1], e[2]);
    e[a] = N;
    const size_t pN = gidx3(g, e[0], e[1], e[2]);
    const int oN = owner_face(g, e[0], e[1], e[2]);
    const bool dir0 = g.bc[o0] == CHEB_DIRICHLET, dirN = g.bc[oN] == CHEB_DIRICHLET;
    const bool neu0 = (o0 == 2 * a + 1) && !dir0;
    const bool neuN = (oN == 2 * a) && !dirN;
    const T r0 = r[p0], rN = r[pN];
    if (lane == 0) {
      if (dir0) x[p0] = r0;
      if (dirN) x[pN] = rN;
    }
    if (!neu0 && !neuN) continue;
    T s0 = 0, sN = 0;
    for (int l = 1 + lane; l < N; l += 32) {
      e[a] = l;
      const T v = x[gidx3(g, e[0], e[1], e[2])];
      s0 += D0[l] * v;
      sN += DN[l] * v;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      s0 += __shfl_down_sync(0xffffffffu, s0, d);
      sN += __shfl_down_sync(0xffffffffu, sN, d);
    }
    if (lane != 0) continue;
    // rows: +(D00 x0 + D0N xN + s0) = r0 ; -(DN0 x0 + DNN xN + sN) = rN
    const T a00 = D0[0], a01 = D0[N], a10 = DN[0], a11 = DN[N];
    const T b0 = r0 - s0, b1 = -rN - sN;
    if (neu0 && neuN) {
      const T det = a00 * a11 - a01 * a10;
      x[p0] = (b0 * a11 - a01 * b1) / det;
      x[pN] = (a00 * b1 - a10 * b0) / det;
    } else if (neu0) {
      const T xN = dirN ? rN : x[pN];
      x[p0] = (b0 - a01 * xN) / a00;
    } else {
      const T x0 = dir0 ? r0 : x[p0];
      x[pN] = (b1 - a10 * x0) / a11;
    }
  }
}
template <typename T>
__global__ void fdm_bline_kernel(Geom g, FdmK<T> t, int a, int kind, const T* __restrict__ r,
                                 T* __restrict__ x) {
  fdm_bline_body(g, t, a, kind, r, x, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// transposed preconditioner M^{-T} (for the adjoint solve): the steps of
// M^{-1} in reverse order, each transposed.  Y is a work copy of the input
// that collects the adjoints of intermediate values; z is the output.
// ---------------------------------------------------------------------------

// Transposed end-row solves on boundary lines (kind 1 or 2, as in
// fdm_bline_kernel): for every end solved from a Neumann row of axis a,
// route its adjoint to z at the two ends and to Y along the line interior.
template <typename T>
__global__ void fdm_bline_t_kernel(Geom g, FdmK<T> t, int a, int kind, T* __restrict__ Y,
                                   T* __restrict__ z) {
  const int nb_axes = g.dim - 1;
  int others[2], no = 0;
  for (int q = 0; q < g.dim; ++q)
    if (q != a) others[no++] = q;
  int total;
  if (kind == 1) {
    int cnt = 0;
    for (int q = 0; q < nb_axes; ++q) {
      const int cax = (nb_axes == 2) ? others[1 - q] : -1;
      cnt += 2 * (cax >= 0 ? g.n[cax] - 2 : 1);
    }
    total = cnt;
  } else {
    total = (nb_axes == 2) ? 4 : 0;
  }
  const int n = g.n[a], N = n - 1;
  const T* D0 = t.Drow[a];
  const T* DN = t.Drow[a] + n;
  for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < total; L += gridDim.x * blockDim.x) {
    int idx[3] = {0, 0, 0};
    if (kind == 1) {
      int rest = L, q = 0;
      for (; q < nb_axes; ++q) {
        const int cax = (nb_axes == 2) ? others[1 - q] : -1;
        const int span = 2 * (cax >= 0 ? g.n[cax] - 2 : 1);
        if (rest < span) break;
        rest -= span;
      }
      const int bax = others[q];
      const int cax = (nb_axes == 2) ? others[1 - q] : -1;
      const int side = rest & 1, tt = rest >> 1;
      idx[bax] = side ? 0 : g.n[bax] - 1;
      if (cax >= 0) idx[cax] = 1 + tt;
    } else {
      idx[others[0]] = (L & 1) ? 0 : g.n[others[0]] - 1;
      idx[others[1]] = (L & 2) ? 0 : g.n[others[1]] - 1;
    }
    int e[3] = {idx[0], idx[1], idx[2]};
    e[a] = 0;
    const size_t p0 = gidx3(g, e[0], e[1], e[2]);
    const int o0 = owner_face(g, e[0], e[1], e[2]);
    e[a] = N;
    const size_t pN = gidx3(g, e[0], e[1], e[2]);
    const int oN = owner_face(g, e[0], e[1], e[2]);
    const bool dir0 = g.bc[o0] == CHEB_DIRICHLET, dirN = g.bc[oN] == CHEB_DIRICHLET;
    const bool neu0 = (o0 == 2 * a + 1) && !dir0;
    const bool neuN = (oN == 2 * a) && !dirN;
    if (!neu0 && !neuN) continue;
    const T a00 = D0[0], a01 = D0[N], a10 = DN[0], a11 = DN[N];
    // adjoints of the right-hand sides b0 = r0 - s0, b1 = -rN - sN
    T bb0 = 0, bb1 = 0;
    if (neu0 && neuN) {
      const T y0 = Y[p0], yN = Y[pN];
      const T det = a00 * a11 - a01 * a10;
      // [b0; b1] = A^{-T} [y0; yN]
      bb0 = (a11 * y0 - a10 * yN) / det;
      bb1 = (-a01 * y0 + a00 * yN) / det;
      z[p0] = bb0;
      z[pN] = -bb1;
    } else if (neu0) {
      // x0 = (b0 - a01 rN) / a00 with rN the Dirichlet value of the other end:
      // that end's adjoint gains -a01 bb0 (its own copy is added later)
      bb0 = Y[p0] / a00;
      z[p0] = bb0;
      Y[pN] -= a01 * bb0;
    } else {
      bb1 = Y[pN] / a11;
      z[pN] = -bb1;
      Y[p0] -= a10 * bb1;
    }
    for (int l = 1; l < N; ++l) {
      e[a] = l;
      Y[gidx3(g, e[0], e[1], e[2])] -= bb0 * D0[l] + bb1 * DN[l];
    }
  }
}

// Dirichlet-owned edge / corner nodes: z = Y (the transposed copy x = r).
template <typename T>
__global__ void fdm_edge_dirichlet_t_kernel(Geom g, const T* __restrict__ Y, T* __restrict__ z) {
  const size_t tot = (size_t)g.n[0] * g.n[1] * g.n[2];
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int k = (int)(c / ((size_t)g.n[0] * g.n[1]));
    const int idx[3] = {i, j, k};
    int nf = 0;
    for (int a = 0; a < g.dim; ++a) nf += (idx[a] == 0 || idx[a] == g.n[a] - 1);
    if (nf < 2) continue;
    const int o = owner_face(g, i, j, k);
    if (g.bc[o] == CHEB_DIRICHLET) z[c] = Y[c];
  }
}

// Transpose of the face step and the interior scatter:
//   Ubar[c] = Y[I(c)] + sum_a (G_a[0][c_a] Y[e0_a(c)] + G_a[1][c_a] Y[eN_a(c)])
template <typename T>
__global__ void fdm_gather_t_kernel(Geom g, FdmK<T> t, const T* __restrict__ Y, T* __restrict__ U) {
  FDM_CELL_INDEX
  {
    const int idx[3] = {ci + t.off[0], cj + t.off[1], ck + t.off[2]};
    const int cl[3] = {ci, cj, ck};
    T v = Y[gidx3(g, idx[0], idx[1], idx[2])];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.dim) break;
      int e0[3] = {idx[0], idx[1], idx[2]}, eN[3] = {idx[0], idx[1], idx[2]};
      e0[a] = 0;
      eN[a] = g.n[a] - 1;
      const int ma = t.m[a];
      v += t.G[a][cl[a]] * Y[gidx3(g, e0[0], e0[1], e0[2])] +
           t.G[a][ma + cl[a]] * Y[gidx3(g, eN[0], eN[1], eN[2])];
    }
    U[cpos(t, ci, cj, ck)] = v;
  }
}

// Per interior a-line: z[e0], z[eN] = Binv^T (Y[e0], Y[eN]) + kref (Lh^T Ubar(line)).
template <typename T>
__global__ void fdm_faces_t_kernel(Geom g, FdmK<T> t, int a, T kref, const T* __restrict__ U,
                                   const T* __restrict__ Y, T* __restrict__ z) {
  const int ma = t.m[a];
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  const size_t lines = (size_t)t.m[b] * t.m[c];
  const size_t str[3] = {1, (size_t)t.mp[0], (size_t)t.mp[0] * t.mp[1]};
  const T* Lh = t.Lh[a];
  const T* Bi = t.Binv[a];
  for (size_t L = blockIdx.x * (size_t)blockDim.x + threadIdx.x; L < lines; L += (size_t)gridDim.x * blockDim.x) {
    const int cb = (int)(L % t.m[b]), cc = (int)(L / t.m[b]);
    int cidx[3];
    cidx[a] = 0; cidx[b] = cb; cidx[c] = cc;
    const size_t base = cidx[0] * str[0] + cidx[1] * str[1] + cidx[2] * str[2];
    T s0 = 0, sN = 0;
    for (int l = 0; l < ma; ++l) {
      const T v = U[base + (size_t)l * str[a]];
      s0 += Lh[l * 2 + 0] * v;
      sN += Lh[l * 2 + 1] * v;
    }
    int idx[3] = {cidx[0] + t.off[0], cidx[1] + t.off[1], cidx[2] + t.off[2]};
    idx[a] = 0;
    const size_t p0 = gidx3(g, idx[0], idx[1], idx[2]);
    idx[a] = g.n[a] - 1;
    const size_t pN = gidx3(g, idx[0], idx[1], idx[2]);
    const T y0 = Y[p0], yN = Y[pN];
    z[p0] = Bi[0] * y0 + Bi[2] * yN + kref * s0;
    z[pN] = Bi[1] * y0 + Bi[3] * yN + kref * sN;
  }
}

template <typename T> static FdmK<T> make_k(const Fdm& f, int dim);
template <> FdmK<double> make_k<double>(const Fdm& f, int dim) {
  FdmK<double> k;
  k.active = f.active;
  for (int a = 0; a < 3; ++a) {
    k.m[a] = f.m[a];
    k.mp[a] = f.mp[a];
    k.off[a] = a < dim ? 1 : 0;
    k.Lh[a] = f.d64[a].Lh; k.lam[a] = f.d64[a].lam; k.G[a] = f.d64[a].G;
    k.Binv[a] = f.d64[a].Binv; k.Drow[a] = f.d64[a].Drow;
  }
  return k;
}
template <> FdmK<float> make_k<float>(const Fdm& f, int dim) {
  FdmK<float> k;
  k.active = f.active;
  for (int a = 0; a < 3; ++a) {
    k.m[a] = f.m[a];
    k.mp[a] = f.mp[a];
    k.off[a] = a < dim ? 1 : 0;
    k.Lh[a] = f.d32[a].Lh; k.lam[a] = f.d32[a].lam; k.G[a] = f.d32[a].G;
    k.Binv[a] = f.d32[a].Binv; k.Drow[a] = f.d32[a].Drow;
  }
  return k;
}

template <typename T> static T** ubuf(Fdm& f);
template <> double** ubuf<double>(Fdm& f) { return f.U64; }
template <> float** ubuf<float>(Fdm& f) { return f.U32; }
template <typename T> static const FdmAxisDev<T>& axdev(const Fdm& f, int a);
template <> const FdmAxisDev<double>& axdev<double>(const Fdm& f, int a) { return f.d64[a]; }
template <> const FdmAxisDev<float>& axdev<float>(const Fdm& f, int a) { return f.d32[a]; }

template <typename T>
static int gemm_any(int M, int N, int K, const T* A, int lda, long long sA, const T* B, int ldb, long long sB,
                    T* C, int ldc, long long sC, int batch, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (tf32x3_ok(K, A, lda, sA, B, ldb, sB))
      return k_gemm_tf32x3(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, s);
  }
  return k_gemm<T>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, s);
}

// out = Mat applied along axis a of the padded compact array `in`
// (out[.., i, ..] = sum_l Mat[i][l] in[.., l, ..]); MatT is Mat transposed.
template <typename T>
static int along(const Fdm& f, int a, const T* Mat, const T* MatT, const T* in, T* out, cudaStream_t s) {
  const int px = f.mp[0], py = f.mp[1], pz = f.mp[2];
  if (a == 0) return gemm_any<T>(py * pz, px, px, in, px, 0, MatT, px, 0, out, px, 0, 1, s);
  if (a == 1)
    return gemm_any<T>(py, px, py, Mat, py, 0, in, px, (long long)py * px, out, px, (long long)py * px, pz, s);
  return gemm_any<T>(pz, py * px, pz, Mat, pz, 0, in, py * px, 0, out, py * px, 0, 1, s);
}

int fdm_clear(const Fdm& f, cudaStream_t s) {
  const size_t ptot = (size_t)f.mp[0] * f.mp[1] * f.mp[2];
  for (int i = 0; i < 2; ++i) {
    if (f.U64[i]) CHEB_CUDA(cudaMemsetAsync(f.U64[i], 0, sizeof(double) * ptot, s));
    if (f.U32[i]) CHEB_CUDA(cudaMemsetAsync(f.U32[i], 0, sizeof(float) * ptot, s));
  }
  return CHEB_OK;
}

template <typename T>
static int ensure_compact(Fdm& f, T** U, cudaStream_t s) {
  if (U[0]) return CHEB_OK;
  const size_t ptot = (size_t)f.mp[0] * f.mp[1] * f.mp[2];
  CHEB_CUDA(cudaMalloc(&U[0], sizeof(T) * ptot));
  CHEB_CUDA(cudaMalloc(&U[1], sizeof(T) * ptot));
  // the padding must read as zero for the contractions and stays zero
  CHEB_CUDA(cudaMemsetAsync(U[0], 0, sizeof(T) * ptot, s));
  CHEB_CUDA(cudaMemsetAsync(U[1], 0, sizeof(T) * ptot, s));
  return CHEB_OK;
}

static int grid_for(size_t n) {
  return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 8));
}

template <typename T>
static bool rotating(const Fdm& f) {
  return sizeof(T) == 4 && f.rot;
}

// Matrix q (0 S, 1 S^{-1}, 2 S^T, 3 S^{-T}) along every axis on the tcgen05
// kernel: each contraction runs along the contiguous axis and writes its
// output transposed, so after dim contractions the layout is restored.  The
// axis products commute, so the sweep order is always x, y, z.  The last
// contraction uses the epilogue `last` (its row decomposition filled here).
static int rot_sweep(const cheb_plan_s* p, Fdm& f, float** U, int& cur, int q, UmmaEpi last,
                     cudaStream_t s) {
  const size_t ptot = (size_t)f.mp[0] * f.mp[1] * f.mp[2];
  const int L = p->dim - 1;
  // rows of the last contraction: [y][x] in 3-D, [x] in 2-D
  last.mpf = f.mp[0];
  last.mf = f.m[0];
  last.ms = p->dim == 3 ? f.m[1] : 1;
  last.mc = f.m[L];
  for (int a = 0; a < p->dim; ++a) {
    const int K = f.mp[a];
    UmmaEpi plain;
    plain.active = f.active;
    last.active = f.active;
    const int st = umma_tf32x3_rot(U[cur], f.uw[a][2 * q], f.tf32_mats ? nullptr : f.uw[a][2 * q + 1], U[1 - cur],
                                   (int)(ptot / K), K, K, a == L ? last : plain, s);
    if (st) return st;
    if (!(a == L && last.mode == 2)) cur = 1 - cur;
  }
  return CHEB_OK;
}

// eigenvalue division fused into the last contraction of the S^{-1} sweep
static UmmaEpi epi_scale(const cheb_plan_s* p, const Fdm& f, double kref) {
  UmmaEpi e;
  e.mode = 1;
  e.lf = f.d32[0].lam;
  e.ls = p->dim == 3 ? f.d32[1].lam : nullptr;
  e.lc = f.d32[p->dim - 1].lam;
  e.kref = (float)kref;
  return e;
}

static dim3 grid3(const Fdm& f) { return dim3((f.m[0] + 127) / 128, f.m[1], f.m[2]); }

// interior of the full grid as a face-step source
template <typename T>
static FdmSrc<T> full_src(const cheb_plan_s* p, const T* x) {
  const long long n0 = p->n[0], n01 = (long long)p->n[0] * (p->dim > 1 ? p->n[1] : 1);
  long long off = 1;
  if (p->dim > 1) off += n0;
  if (p->dim > 2) off += n01;
  return FdmSrc<T>{x, off, n0, n01};
}

// Face end values of the interior lines of axes [a0, a1), then the
// boundary-line solves (edges, axis by axis, then corners).
template <typename T>
static int faces_and_blines(const cheb_plan_s* p, const Fdm& f, const FdmK<T>& k, FdmSrc<T> u, int a0, int a1,
                            const T* r, T* x, cudaStream_t s) {
  const Geom g = p->geom();
  for (int a = a0; a < a1; ++a) {
    if (a == 0) {
      const size_t lines = (size_t)f.m[1] * f.m[2];
      fdm_faces_x_kernel<T><<<grid_for(lines * 32), 256, 0, s>>>(g, k, u, r, x);
    } else {
      const dim3 grid((f.m[0] + 31) / 32, a == 1 ? f.m[2] : f.m[1]);
      fdm_faces_yz_kernel<T><<<grid, 256, 0, s>>>(g, k, a, u, r, x);
    }
    CHEB_LAUNCH_CHECK("fdm_faces_kernel");
  }
  if (p->dim >= 2) {
    for (int a = 0; a < p->dim; ++a) {
      fdm_bline_kernel<T><<<64, 256, 0, s>>>(g, k, a, 1, r, x);
      CHEB_LAUNCH_CHECK("fdm_bline_kernel");
    }
  }
  if (p->dim == 3) {
    for (int a = 0; a < 3; ++a) {
      fdm_bline_kernel<T><<<1, 128, 0, s>>>(g, k, a, 2, r, x);
      CHEB_LAUNCH_CHECK("fdm_bline_kernel");
    }
  }
  return CHEB_OK;
}


template <typename T> static T* ybuf(Fdm& f);
template <> double* ybuf<double>(Fdm& f) { return f.Y64; }
template <> float* ybuf<float>(Fdm& f) { return f.Y32; }

template <typename T>
static int ensure_ybuf(const cheb_plan_s* p, Fdm& f) {
  if (ybuf<T>(f)) return CHEB_OK;
  T* yb = nullptr;
  CHEB_CUDA(cudaMalloc(&yb, sizeof(T) * p->size()));
  if constexpr (sizeof(T) == 8) f.Y64 = (double*)yb;
  else f.Y32 = (float*)yb;
  return CHEB_OK;
}

// out = in with the values at flux-owned boundary nodes multiplied by fac
// (in and out may alias).  A flux row -kref s (d_a u) = r_p of the
// constant-coefficient operator is the Neumann row s (d_a u) = -r_p / kref.
template <typename T>
__global__ void fdm_flux_scale_kernel(Geom g, T fac, const T* in, T* out) {
  const size_t tot = (size_t)g.n[0] * g.n[1] * g.n[2];
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int kk = (int)(c / ((size_t)g.n[0] * g.n[1]));
    const int o = owner_face(g, i, j, kk);
    const T v = in[c];
    out[c] = (o >= 0 && g.bc[o] == CHEB_FLUX) ? fac * v : v;
  }
}

template <typename T>
int fdm_fill_boundary(const cheb_plan_s* p, Fdm& f, const T* r, T* x, cudaStream_t s) {
  const FdmK<T> k = make_k<T>(f, p->dim);
  return faces_and_blines<T>(p, f, k, full_src<T>(p, x), 0, p->dim, r, x, s);
}
template int fdm_fill_boundary<double>(const cheb_plan_s*, Fdm&, const double*, double*, cudaStream_t);
template int fdm_fill_boundary<float>(const cheb_plan_s*, Fdm&, const float*, float*, cudaStream_t);

template <typename T>
int fdm_apply(const cheb_plan_s* p, Fdm& f, double kref, const T* r, T* x, cudaStream_t s) {
  const Geom g = p->geom();
  const FdmK<T> k = make_k<T>(f, p->dim);
  T** U = ubuf<T>(f);
  int st;
  if ((st = ensure_compact<T>(f, U, s))) return st;
  if (has_flux(p)) {
    // M^{-1} with flux rows = (Neumann-row inverse) after scaling the flux data
    if ((st = ensure_ybuf<T>(p, f))) return st;
    fdm_flux_scale_kernel<T><<<grid_for(p->size()), 256, 0, s>>>(g, (T)(-1.0 / kref), r, ybuf<T>(f));
    CHEB_LAUNCH_CHECK("fdm_flux_scale_kernel");
    r = ybuf<T>(f);
  }
  fdm_lift_kernel<T><<<dim3((f.m[0] + 127) / 128, f.m[1], (f.m[2] + kLiftK - 1) / kLiftK), 128, 0, s>>>(
      g, k, (T)kref, r, U[0]);
  CHEB_LAUNCH_CHECK("fdm_lift_kernel");
  int cur = 0;
  if constexpr (sizeof(T) == 4) {
    if (f.rot) {
      // S^{-1} sweep with the eigenvalue division fused into its last
      // contraction; S sweep whose last contraction writes the interior of
      // x and the end values of the last axis' lines
      if ((st = rot_sweep(p, f, U, cur, 1, epi_scale(p, f, kref), s))) return st;
      UmmaEpi e;
      e.mode = 2;
      const FdmSrc<T> xs = full_src<T>(p, x);
      const int L = p->dim - 1;
      e.x = x;
      e.r = r;
      e.xoff = xs.off;
      e.xs_f = 1;
      e.xs_s = xs.s1;
      e.xs_c = L == 2 ? xs.s2 : xs.s1;
      e.ncol = p->n[L];
      e.G = f.d32[L].G;
      e.Binv = f.d32[L].Binv;
      if ((st = rot_sweep(p, f, U, cur, 0, e, s))) return st;
      return faces_and_blines<T>(p, f, k, xs, 0, L, r, x, s);
    }
  }
  auto contract = [&](int a, bool inverse) -> int {
    const FdmAxisDev<T>& d = axdev<T>(f, a);
    const int rc = inverse ? along<T>(f, a, d.Sinv, d.SinvT, U[cur], U[1 - cur], s)
                           : along<T>(f, a, d.S, d.ST, U[cur], U[1 - cur], s);
    cur = 1 - cur;
    return rc;
  };
  for (int a = 0; a < p->dim; ++a)
    if ((st = contract(a, true))) return st;
  fdm_scale_kernel<T><<<grid3(f), 128, 0, s>>>(k, p->dim, (T)kref, U[cur]);
  CHEB_LAUNCH_CHECK("fdm_scale_kernel");
  for (int a = p->dim - 1; a >= 0; --a)
    if ((st = contract(a, false))) return st;
  fdm_scatter_kernel<T><<<grid3(f), 128, 0, s>>>(g, k, U[cur], x);
  CHEB_LAUNCH_CHECK("fdm_scatter_kernel");
  const FdmSrc<T> us{U[cur], 0, f.mp[0], (long long)f.mp[0] * f.mp[1]};
  return faces_and_blines<T>(p, f, k, us, 0, p->dim, r, x, s);
}

template int fdm_apply<double>(const cheb_plan_s*, Fdm&, double, const double*, double*, cudaStream_t);
template int fdm_apply<float>(const cheb_plan_s*, Fdm&, double, const float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// Batched preconditioner steps of lockstep batch solves: the lift, the face
// steps and the boundary-line passes of several instances in one launch
// each, over a work list of (instance, block) items; each instance's two
// tcgen05 sweeps (fdm_rot_core) run between them.  The split is that of
// the FP32 tcgen05 path of fdm_apply: lift, sweep S^{-1} (eigenvalue
// division fused), sweep S (the last axis' end values written by its
// epilogue), faces of the other axes, boundary lines.
// ---------------------------------------------------------------------------
struct FdmBItem {
  Geom g;
  FdmK<float> k;
  float kref;
  long long off;                   // offset of the instance in the batch vectors
  float* U0;                       // its compact work array (lift output)
  long long xs_off, xs_s1, xs_s2;  // interior of x as face-step source, relative to x + off
  int lgx, lgy, lgz;               // lift grid
  int fx_blocks;                   // face step of axis 0: blocks
  int fy_gx, fy_gy;                // face step of axis 1 (3-D): grid
};

struct FdmBatch {
  int count = 0, dim = 3;
  std::vector<FdmBItem> h;
  FdmBItem* d_items = nullptr;
  int* d_pref[4] = {nullptr, nullptr, nullptr, nullptr};  // lift, faces, lines kind 1, kind 2
  int nblk[4] = {0, 0, 0, 0};
};

bool fdm_batchable(const cheb_plan_s* p, const Fdm& f) {
  return f.ready && f.rot && !has_flux(p) && p->dim >= 2 && f.U32[0] != nullptr;
}

// item of block b: the last i with pref[i] <= b
__device__ __forceinline__ int fdm_item_of(const int* __restrict__ pref, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128) fdm_lift_batch_kernel(const FdmBItem* __restrict__ items,
                                                             const int* __restrict__ pref, int count,
                                                             const float* __restrict__ rb) {
  const int i = fdm_item_of(pref, count, blockIdx.x);
  const FdmBItem& it = items[i];
  const int lb = blockIdx.x - pref[i];
  const int bx = lb % it.lgx, by = (lb / it.lgx) % it.lgy, bz = lb / (it.lgx * it.lgy);
  fdm_lift_body<float>(it.g, it.k, it.kref, rb + it.off, it.U0, bx, by, bz);
}

__global__ void __launch_bounds__(256) fdm_faces_batch_kernel(const FdmBItem* __restrict__ items,
                                                              const int* __restrict__ pref, int count,
                                                              const float* __restrict__ rb, float* __restrict__ xb) {
  const int i = fdm_item_of(pref, count, blockIdx.x);
  const FdmBItem& it = items[i];
  const int lb = blockIdx.x - pref[i];
  float* x = xb + it.off;
  const FdmSrc<float> u{x, it.xs_off, it.xs_s1, it.xs_s2};
  // the two face steps write disjoint nodes and read only interior nodes
  if (lb < it.fx_blocks) {
    fdm_faces_x_body<float>(it.g, it.k, u, rb + it.off, x, lb, it.fx_blocks);
  } else {
    const int q = lb - it.fx_blocks;
    fdm_faces_yz_body<float>(it.g, it.k, 1, u, rb + it.off, x, q % it.fy_gx, q / it.fy_gx);
  }
}

__global__ void __launch_bounds__(256) fdm_bline_batch_kernel(const FdmBItem* __restrict__ items,
                                                              const int* __restrict__ pref, int count, int a,
                                                              int kind, const float* __restrict__ rb,
                                                              float* __restrict__ xb) {
  const int i = fdm_item_of(pref, count, blockIdx.x);
  const FdmBItem& it = items[i];
  fdm_bline_body<float>(it.g, it.k, a, kind, rb + it.off, xb + it.off, blockIdx.x - pref[i],
                        pref[i + 1] - pref[i]);
}

int fdm_batch_create(FdmBatch** out, const std::vector<const cheb_plan_s*>& plans, const std::vector<Fdm*>& fdms,
                     const std::vector<long long>& off) {
  FdmBatch* b = new FdmBatch();
  auto fail = [&](int st) { fdm_batch_free(b); return st; };
  b->count = (int)plans.size();
  if (b->count == 0) { *out = b; return CHEB_OK; }
  b->dim = plans[0]->dim;
  b->h.resize(b->count);
  std::vector<int> pref[4];
  for (auto& v : pref) v.assign(1, 0);
  for (int i = 0; i < b->count; ++i) {
    const cheb_plan_s* p = plans[i];
    Fdm& f = *fdms[i];
    if (!fdm_batchable(p, f) || p->dim != b->dim) { set_error("instance not batchable"); return fail(CHEB_ERR_ARG); }
    FdmBItem& it = b->h[i];
    std::memset(&it, 0, sizeof(it));
    it.g = p->geom();
    it.k = make_k<float>(f, p->dim);
    it.kref = 1.f;
    it.off = off[i];
    it.U0 = f.U32[0];
    const FdmSrc<float> xs = full_src<float>(p, (const float*)nullptr);
    it.xs_off = xs.off;
    it.xs_s1 = xs.s1;
    it.xs_s2 = xs.s2;
    it.lgx = (f.m[0] + 127) / 128;
    it.lgy = f.m[1];
    it.lgz = (f.m[2] + kLiftK - 1) / kLiftK;
    it.fx_blocks = grid_for((size_t)f.m[1] * f.m[2] * 32);
    if (p->dim == 3) {
      it.fy_gx = (f.m[0] + 31) / 32;
      it.fy_gy = f.m[2];
    } else {
      it.fy_gx = 1;
      it.fy_gy = 0;
    }
    pref[0].push_back(pref[0].back() + it.lgx * it.lgy * it.lgz);
    pref[1].push_back(pref[1].back() + it.fx_blocks + it.fy_gx * it.fy_gy);
    pref[2].push_back(pref[2].back() + 64);
    pref[3].push_back(pref[3].back() + 1);
  }
  if (cudaMalloc(&b->d_items, sizeof(FdmBItem) * b->count) != cudaSuccess) return fail(CHEB_ERR_NOMEM);
  if (cudaMemcpy(b->d_items, b->h.data(), sizeof(FdmBItem) * b->count, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(CHEB_ERR_CUDA);
  for (int q = 0; q < 4; ++q) {
    b->nblk[q] = pref[q].back();
    if (cudaMalloc(&b->d_pref[q], sizeof(int) * pref[q].size()) != cudaSuccess) return fail(CHEB_ERR_NOMEM);
    if (cudaMemcpy(b->d_pref[q], pref[q].data(), sizeof(int) * pref[q].size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return fail(CHEB_ERR_CUDA);
  }
  *out = b;
  return CHEB_OK;
}

int fdm_batch_kref(FdmBatch* b, const std::vector<double>& kref) {
  if (!b || b->count == 0) return CHEB_OK;
  for (int i = 0; i < b->count; ++i) b->h[i].kref = (float)kref[i];
  CHEB_CUDA(cudaMemcpy(b->d_items, b->h.data(), sizeof(FdmBItem) * b->count, cudaMemcpyHostToDevice));
  return CHEB_OK;
}

void fdm_batch_free(FdmBatch* b) {
  if (!b) return;
  cudaFree(b->d_items);
  for (auto* p : b->d_pref) cudaFree(p);
  delete b;
}

int fdm_batch_lift(const FdmBatch* b, const float* rb, cudaStream_t s) {
  if (!b || b->count == 0) return CHEB_OK;
  fdm_lift_batch_kernel<<<b->nblk[0], 128, 0, s>>>(b->d_items, b->d_pref[0], b->count, rb);
  CHEB_LAUNCH_CHECK("fdm_lift_batch_kernel");
  return CHEB_OK;
}

int fdm_batch_faces(const FdmBatch* b, const float* rb, float* xb, cudaStream_t s) {
  if (!b || b->count == 0) return CHEB_OK;
  fdm_faces_batch_kernel<<<b->nblk[1], 256, 0, s>>>(b->d_items, b->d_pref[1], b->count, rb, xb);
  CHEB_LAUNCH_CHECK("fdm_faces_batch_kernel");
  // boundary lines: axes in increasing order (an a-line may read an end a lower axis solved)
  for (int a = 0; a < b->dim; ++a) {
    fdm_bline_batch_kernel<<<b->nblk[2], 256, 0, s>>>(b->d_items, b->d_pref[2], b->count, a, 1, rb, xb);
    CHEB_LAUNCH_CHECK("fdm_bline_batch_kernel");
  }
  if (b->dim == 3)
    for (int a = 0; a < 3; ++a) {
      fdm_bline_batch_kernel<<<b->nblk[3], 256, 0, s>>>(b->d_items, b->d_pref[3], b->count, a, 2, rb, xb);
      CHEB_LAUNCH_CHECK("fdm_bline_batch_kernel");
    }
  return CHEB_OK;
}

// the two tcgen05 sweeps of the FP32 path, after the lift wrote U[0]
int fdm_rot_core(const cheb_plan_s* p, Fdm& f, double kref, const float* r, float* x, cudaStream_t s) {
  float** U = ubuf<float>(f);
  int cur = 0, st;
  if ((st = rot_sweep(p, f, U, cur, 1, epi_scale(p, f, kref), s))) return st;
  UmmaEpi e;
  e.mode = 2;
  const FdmSrc<float> xs = full_src<float>(p, x);
  const int L = p->dim - 1;
  e.x = x;
  e.r = r;
  e.xoff = xs.off;
  e.xs_f = 1;
  e.xs_s = xs.s1;
  e.xs_c = L == 2 ? xs.s2 : xs.s1;
  e.ncol = p->n[L];
  e.G = f.d32[L].G;
  e.Binv = f.d32[L].Binv;
  return rot_sweep(p, f, U, cur, 0, e, s);
}

template <typename T>
int fdm_prepare(const cheb_plan_s* p, Fdm& f, cudaStream_t s) {
  int st;
  if ((st = ensure_compact<T>(f, ubuf<T>(f), s))) return st;
  if (has_flux(p) && (st = ensure_ybuf<T>(p, f))) return st;
  return CHEB_OK;
}
template int fdm_prepare<double>(const cheb_plan_s*, Fdm&, cudaStream_t);
template int fdm_prepare<float>(const cheb_plan_s*, Fdm&, cudaStream_t);

template <typename T>
int fdm_apply_t(const cheb_plan_s* p, Fdm& f, double kref, const T* y, T* z, cudaStream_t s) {
  const Geom g = p->geom();
  const FdmK<T> k = make_k<T>(f, p->dim);
  const size_t tot = (size_t)f.m[0] * f.m[1] * f.m[2];
  const size_t nfull = p->size();
  T** U = ubuf<T>(f);
  {
    int st0 = ensure_compact<T>(f, U, s);
    if (st0) return st0;
  }
  {
    int st0 = ensure_ybuf<T>(p, f);
    if (st0) return st0;
  }
  T* Y = ybuf<T>(f);
  CHEB_CUDA(cudaMemcpyAsync(Y, y, sizeof(T) * nfull, cudaMemcpyDeviceToDevice, s));
  if (p->dim == 3) {
    for (int a = 2; a >= 0; --a) {
      fdm_bline_t_kernel<T><<<1, 32, 0, s>>>(g, k, a, 2, Y, z);
      CHEB_LAUNCH_CHECK("fdm_bline_t_kernel");
    }
  }
  if (p->dim >= 2) {
    for (int a = p->dim - 1; a >= 0; --a) {
      fdm_bline_t_kernel<T><<<8, 128, 0, s>>>(g, k, a, 1, Y, z);
      CHEB_LAUNCH_CHECK("fdm_bline_t_kernel");
    }
    fdm_edge_dirichlet_t_kernel<T><<<grid_for(nfull), 256, 0, s>>>(g, Y, z);
    CHEB_LAUNCH_CHECK("fdm_edge_dirichlet_t_kernel");
  }
  fdm_gather_t_kernel<T><<<grid3(f), 128, 0, s>>>(g, k, Y, U[0]);
  CHEB_LAUNCH_CHECK("fdm_gather_t_kernel");
  int cur = 0;
  // (S_all Lambda^{-1} Sinv_all)^T = Sinv_all^T Lambda^{-1} S_all^T
  auto contract_t = [&](int a, bool inverse) -> int {
    const FdmAxisDev<T>& d = axdev<T>(f, a);
    const int rc = inverse ? along<T>(f, a, d.SinvT, d.Sinv, U[cur], U[1 - cur], s)
                           : along<T>(f, a, d.ST, d.S, U[cur], U[1 - cur], s);
    cur = 1 - cur;
    return rc;
  };
  int st;
  if (rotating<T>(f)) {
    // S^T sweep with the eigenvalue division fused, then the S^{-T} sweep
    if ((st = rot_sweep(p, f, (float**)U, cur, 2, epi_scale(p, f, kref), s))) return st;
    if ((st = rot_sweep(p, f, (float**)U, cur, 3, UmmaEpi(), s))) return st;
  } else {
    for (int a = 0; a < p->dim; ++a)
      if ((st = contract_t(a, false))) return st;
    fdm_scale_kernel<T><<<grid3(f), 128, 0, s>>>(k, p->dim, (T)kref, U[cur]);
    CHEB_LAUNCH_CHECK("fdm_scale_kernel");
    for (int a = p->dim - 1; a >= 0; --a)
      if ((st = contract_t(a, true))) return st;
  }
  fdm_scatter_kernel<T><<<grid3(f), 128, 0, s>>>(g, k, U[cur], z);
  CHEB_LAUNCH_CHECK("fdm_scatter_kernel");
  for (int a = 0; a < p->dim; ++a) {
    const size_t lines = tot / f.m[a];
    fdm_faces_t_kernel<T><<<grid_for(lines), 256, 0, s>>>(g, k, a, (T)kref, U[cur], Y, z);
    CHEB_LAUNCH_CHECK("fdm_faces_t_kernel");
  }
  if (has_flux(p)) {
    // (M_N^{-1} S)^T with S the flux-row scaling = S M_N^{-T}
    fdm_flux_scale_kernel<T><<<grid_for(nfull), 256, 0, s>>>(g, (T)(-1.0 / kref), z, z);
    CHEB_LAUNCH_CHECK("fdm_flux_scale_kernel");
  }
  return CHEB_OK;
}

template int fdm_apply_t<double>(const cheb_plan_s*, Fdm&, double, const double*, double*, cudaStream_t);
template int fdm_apply_t<float>(const cheb_plan_s*, Fdm&, double, const float*, float*, cudaStream_t);

}  // namespace cheb
