// Line-pass building blocks shared by the line-pass translation units
// (apply.cu: power-of-two transform route and dense route; chirp.cu: the
// transform route for any N): per-axis kernel tables, the tile <-> global
// mapping, the per-warp transform derivative, the block-wide dense
// derivative and the generic line-pass kernel.
#pragma once

#include "device.cuh"
#include "internal.h"

namespace cheb {

template <typename T>
struct AxisK {
  int n, N;
  T scale;
  const typename C2<T>::t* tw;     // P stage twiddles of the warp FFT (transform route)
  const typename C2<T>::t* chirp;  // chirp route: c_j, j < 2N (null: P = 2N, plain FFT)
  const typename C2<T>::t* bhat;   // chirp route: transformed convolution kernel (P)
  const T* D;                      // n x n row-major (dense route)
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory layout of a line pass: X (tile), ends (2 x TL x 2),
// then the route's buffers.  The transform route of this kernel is the
// chirp form (any N): one padded length-P buffer per warp, then the stage
// twiddles (P), the chirp (P / 2 >= 2N) and the kernel transform (P).
template <typename T>
static size_t pass_smem_bytes(int route, int n, int P, int TL) {
  const int ldx = n | 1;
  size_t b = align16(sizeof(T) * TL * ldx) + align16(sizeof(T) * TL * 4);
  if (route == CHEB_ROUTE_TRANSFORM) {
    const size_t bl = (size_t)P + P / 8;  // FftBuf<P>::len
    b += align16(2 * sizeof(T) * (size_t)(TL / 2) * bl) + align16(2 * sizeof(T) * (size_t)P) +
         align16(2 * sizeof(T) * (size_t)(P / 2)) + align16(2 * sizeof(T) * (size_t)P);
  } else {
    b += align16(sizeof(T) * TL * ldx) + align16(sizeof(T) * (size_t)n * n);
  }
  return b;
}

// Tile <-> global mapping of element (lane l, point pt).
struct TileMap {
  int axis, nx, ny, nz, TL;
  int line0;      // axis 0: first line of the tile
  int i0, outer;  // axes 1, 2: first x index, fixed k (axis 1) or j (axis 2)
  __device__ __forceinline__ bool at(int l, int pt, size_t& gidx, int& i, int& j, int& k) const {
    if (axis == 0) {
      const int line = line0 + l;
      if (line >= ny * nz) return false;
      i = pt; j = line % ny; k = line / ny;
      gidx = (size_t)line * nx + pt;
    } else {
      i = i0 + l;
      if (i >= nx) return false;
      if (axis == 1) { j = pt; k = outer; }
      else { j = outer; k = pt; }
      gidx = ((size_t)k * ny + j) * nx + i;
    }
    return true;
  }
  // element e of the tile in a coalesced enumeration order
  __device__ __forceinline__ void split(int e, int n, int& l, int& pt) const {
    if (axis == 0) { l = e / n; pt = e - l * n; }
    else { pt = e / TL; l = e - pt * TL; }
  }
};

// ---------------------------------------------------------------------------
// per-warp transform derivative of lines 2w, 2w+1 (in place in X)
// ---------------------------------------------------------------------------
// CHIRP: the length-2N DFT runs as Bluestein's convolution of FFT length P
// (any N); otherwise P = 2N and it is one warp FFT.
template <typename T, int P, int CM, bool TRANSPOSE, bool CHIRP = false>
__device__ __forceinline__ void warp_deriv_tf(T* X, int ldx, typename C2<T>::t* buf,
                                              const typename C2<T>::t* tw, int N, T scale,
                                              int w, int lane,
                                              const typename C2<T>::t* chirp = nullptr,
                                              const typename C2<T>::t* bhat = nullptr) {
  typedef typename C2<T>::t C;
  T* xa = X + (2 * w) * ldx;
  T* xb = X + (2 * w + 1) * ldx;
  const T invN = (T)1 / (T)N;
  const int M = 2 * N;  // length of the even extension
  // weight m_j of the DCT-I matrix columns: 1 at the ends, 2 inside
  auto pack = [&](bool divide_m) {
    for (int j = lane; j < M; j += 32) {
      const int jj = j <= N ? j : M - j;
      C v;
      v.x = xa[jj];
      v.y = xb[jj];
      if (divide_m && jj != 0 && jj != N) { v.x *= (T)0.5; v.y *= (T)0.5; }
      buf[fpad(j)] = v;
    }
    __syncwarp();
  };
  auto weight = [&](int k) -> T {  // w_k = k c_k scale / N
    T wk = (T)k * scale * invN;
    return k == N ? (T)0.5 * wk : wk;
  };
  if (!TRANSPOSE) {
    pack(false);
    if constexpr (CHIRP) warp_dft_chirp<T, P>(buf, tw, chirp, bhat, M, lane);
    else warp_fft<T, P>(buf, tw, lane);
    for (int k = lane; k <= N; k += 32) {
      const T wk = weight(k);
      const C F = buf[fpad(k)];
      xa[k] = wk * F.x;
      xb[k] = wk * F.y;
    }
    __syncwarp();
    warp_parity_scan<T, CM, true>(xa, N, lane);
    warp_parity_scan<T, CM, true>(xb, N, lane);
    pack(false);
    if constexpr (CHIRP) warp_dft_chirp<T, P>(buf, tw, chirp, bhat, M, lane);
    else warp_fft<T, P>(buf, tw, lane);
    for (int k = lane; k <= N; k += 32) {
      const C F = buf[fpad(k)];
      xa[k] = F.x;
      xb[k] = F.y;
    }
    __syncwarp();
  } else {
    // D^T = diag(m) M diag(1/m) W S^T diag(m) M diag(1/m), M = DCT-I matrix,
    // S^T the exclusive parity prefix scan.
    pack(true);
    if constexpr (CHIRP) warp_dft_chirp<T, P>(buf, tw, chirp, bhat, M, lane);
    else warp_fft<T, P>(buf, tw, lane);
    for (int k = lane; k <= N; k += 32) {
      const T mk = (k == 0 || k == N) ? (T)1 : (T)2;
      const C F = buf[fpad(k)];
      xa[k] = mk * F.x;
      xb[k] = mk * F.y;
    }
    __syncwarp();
    warp_parity_scan<T, CM, false>(xa, N, lane);
    warp_parity_scan<T, CM, false>(xb, N, lane);
    for (int k = lane; k <= N; k += 32) {
      const T wk = weight(k);
      xa[k] *= wk;
      xb[k] *= wk;
    }
    __syncwarp();
    pack(true);
    if constexpr (CHIRP) warp_dft_chirp<T, P>(buf, tw, chirp, bhat, M, lane);
    else warp_fft<T, P>(buf, tw, lane);
    for (int k = lane; k <= N; k += 32) {
      const T mk = (k == 0 || k == N) ? (T)1 : (T)2;
      const C F = buf[fpad(k)];
      xa[k] = mk * F.x;
      xb[k] = mk * F.y;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// block-wide dense derivative X <- D X (or D^T X), tile lines as rows.
// FP32 (shared-memory bound): a work item is 2 points x 4 lines (8
// accumulators); consecutive threads take the 4-line groups of one point
// pair, then the next pair, so a warp reads 8 rows of D (odd n: distinct
// banks, each broadcast to 4 threads) and 4 rows of the tile per point m:
// 6 shared-memory wavefronts per 256 FMAs (the 1-point items below: 5 per
// 128).  FP64 (FP64-pipe bound) keeps 1 point x 4 lines per item, twice the
// items, so small n still fills the CTA.  Measured (FP32 / FP64 dense apply):
// 97^3 0.175 -> 0.143 ms with 2-point items; FP64 with them 33^3 +39 %,
// 129^3 +17 %.
// ---------------------------------------------------------------------------
template <typename T, bool TRANSPOSE, int TL>
__device__ __forceinline__ void block_deriv_dense(T* X, T* tmp, int ldx, const T* Dm, int n) {
  constexpr int G = 4;  // lines per work item
  if constexpr (sizeof(T) == 4) {
    constexpr int NLG = TL / G;   // line groups of the tile
    const int np = (n + 1) >> 1;  // point pairs
    const int items = np * NLG;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int l0 = (it % NLG) * G;
      const int i0 = 2 * (it / NLG);
      const bool two = i0 + 1 < n;
      const int i1 = two ? i0 + 1 : i0;  // odd n: the last pair repeats its point (dropped)
      T a0[G], a1[G];
#pragma unroll
      for (int g = 0; g < G; ++g) { a0[g] = (T)0; a1[g] = (T)0; }
      for (int m = 0; m < n; ++m) {
        const T d0 = TRANSPOSE ? Dm[m * n + i0] : Dm[i0 * n + m];
        const T d1 = TRANSPOSE ? Dm[m * n + i1] : Dm[i1 * n + m];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const T x = X[(l0 + g) * ldx + m];
          a0[g] += d0 * x;
          a1[g] += d1 * x;
        }
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        tmp[(l0 + g) * ldx + i0] = a0[g];
        if (two) tmp[(l0 + g) * ldx + i0 + 1] = a1[g];
      }
    }
  } else {
    const int items = n * (TL / G);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int i = it % n;
      const int l0 = (it / n) * G;
      T acc[G];
#pragma unroll
      for (int g = 0; g < G; ++g) acc[g] = (T)0;
      for (int m = 0; m < n; ++m) {
        const T d = TRANSPOSE ? Dm[m * n + i] : Dm[i * n + m];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] += d * X[(l0 + g) * ldx + m];
      }
#pragma unroll
      for (int g = 0; g < G; ++g) tmp[(l0 + g) * ldx + i] = acc[g];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TL * ldx; e += blockDim.x) X[e] = tmp[e];
  __syncthreads();
}

// The transform route here is the chirp form (power-of-two N runs the
// compile-time-N tf_pass_kernel instead).
template <typename T, int ROUTE, int P, int CM, bool TRANSPOSE, int TL>
__device__ __forceinline__ void tile_deriv(T* X, T* tmp, int ldx, typename C2<T>::t* Cb,
                                           const typename C2<T>::t* tw, const T* Dm, int n,
                                           T scale, const typename C2<T>::t* chirp,
                                           const typename C2<T>::t* bhat) {
  if constexpr (ROUTE == CHEB_ROUTE_TRANSFORM) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    warp_deriv_tf<T, P, CM, TRANSPOSE, true>(X, ldx, Cb + (size_t)w * FftBuf<P>::len, tw, n - 1, scale, w,
                                             lane, chirp, bhat);
    __syncthreads();
  } else {
    __syncthreads();
    block_deriv_dense<T, TRANSPOSE, TL>(X, tmp, ldx, Dm, n);
  }
}

// chirp-form passes (chirp.cu); P = the axis' convolution length
template <typename T>
int launch_chirp_pass(const Geom& g, int axis, int kind, const AxisK<T>& ak, int P, const T* K,
                      const T* u, T* out, cudaStream_t s, const T* C);

// ---------------------------------------------------------------------------
// the line-pass kernel
// ---------------------------------------------------------------------------
// Shared-memory pointers of one line pass (layout of pass_smem_bytes).
template <typename T>
struct PassSmem {
  T* X;
  T* ends;
  typename C2<T>::t *Cb, *tw, *ch, *bh;
  T *tmp, *Dm;
};

// Carve the pass' shared memory for the axis tables `ax` and stage the
// tables (chirp transform: twiddles, chirp, kernel transform; dense: D).
// The caller synchronises before the tables are read.
template <typename T, int ROUTE, int P, int TL>
__device__ __forceinline__ PassSmem<T> pass_stage(unsigned char* p, const AxisK<T>& ax) {
  typedef typename C2<T>::t C;
  const int n = ax.n, N = ax.N;
  const int ldx = n | 1;
  PassSmem<T> sm;
  sm.X = (T*)p;            p += align16(sizeof(T) * TL * ldx);
  sm.ends = (T*)p;         p += align16(sizeof(T) * TL * 4);
  sm.Cb = sm.tw = sm.ch = sm.bh = nullptr;
  sm.tmp = sm.Dm = nullptr;
  if (ROUTE == CHEB_ROUTE_TRANSFORM) {
    sm.Cb = (C*)p;         p += align16(2 * sizeof(T) * (size_t)(TL / 2) * FftBuf<P>::len);
    sm.tw = (C*)p;         p += align16(2 * sizeof(T) * (size_t)P);
    sm.ch = (C*)p;         p += align16(2 * sizeof(T) * (size_t)(P / 2));
    sm.bh = (C*)p;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
      sm.tw[t] = ax.tw[t];
      sm.bh[t] = ax.bhat[t];
    }
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) sm.ch[t] = ax.chirp[t];
  } else {
    sm.tmp = (T*)p;        p += align16(sizeof(T) * TL * ldx);
    sm.Dm = (T*)p;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sm.Dm[t] = ax.D[t];
  }
  return sm;
}

// One tile of TL lines of a line pass (tile index `tile` of the axis'
// tiling: x lines in groups of TL, y / z lines in TL-wide x blocks).
template <typename T, int ROUTE, int P, int CM, int TL>
__device__ __forceinline__ void line_pass_tile(const Geom& g, int axis, int kind, const AxisK<T>& ax,
                                               const T* __restrict__ K, const T* __restrict__ u,
                                               T* __restrict__ out, const T* __restrict__ Cj, int tile,
                                               const PassSmem<T>& sm) {
  typedef typename C2<T>::t C;
  const int n = ax.n, N = ax.N;
  const int ldx = n | 1;
  T* X = sm.X;
  T* ends = sm.ends;
  C* Cb = sm.Cb;
  const C* tw = sm.tw;
  const C* ch = sm.ch;
  const C* bh = sm.bh;
  T* tmp = sm.tmp;
  const T* Dm = sm.Dm;
  TileMap map;
  map.axis = axis; map.nx = g.n[0]; map.ny = g.n[1]; map.nz = g.n[2]; map.TL = TL;
  if (axis == 0) {
    map.line0 = tile * TL; map.i0 = 0; map.outer = 0;
  } else {
    const int nbx = (g.n[0] + TL - 1) / TL;
    map.line0 = 0;
    map.i0 = (tile % nbx) * TL;
    map.outer = tile / nbx;
  }
  const int tile_elems = TL * n;

  // load the input tile (u, or lambda for the adjoint)
  for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
    int l, pt; map.split(e, n, l, pt);
    size_t gi; int i, j, k;
    T v = (T)0;
    if (map.at(l, pt, gi, i, j, k)) v = u[gi];
    X[l * ldx + pt] = v;
  }
  __syncthreads();

  const bool adj = (kind == kAdjFirst || kind == kAdjAcc);
  if (kind == kDeriv || kind == kDerivT) {
    if (kind == kDeriv) tile_deriv<T, ROUTE, P, CM, false, TL>(X, tmp, ldx, Cb, tw, Dm, n, ax.scale, ch, bh);
    else tile_deriv<T, ROUTE, P, CM, true, TL>(X, tmp, ldx, Cb, tw, Dm, n, ax.scale, ch, bh);
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
      int l, pt; map.split(e, n, l, pt);
      size_t gi; int i, j, k;
      if (map.at(l, pt, gi, i, j, k)) out[gi] = X[l * ldx + pt];
    }
    return;
  }

  if (!adj) {
    // ---- A u (or the Jacobian action): D_a u, keep line-end derivatives for
    // Neumann rows; after the product q = K D_a u (+ C u) keep its line-end
    // values for flux rows (-s q at the owner face)
    tile_deriv<T, ROUTE, P, CM, false, TL>(X, tmp, ldx, Cb, tw, Dm, n, ax.scale, ch, bh);
    if (threadIdx.x < TL) {
      ends[threadIdx.x * 2 + 0] = X[threadIdx.x * ldx + 0];
      ends[threadIdx.x * 2 + 1] = X[threadIdx.x * ldx + N];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
      int l, pt; map.split(e, n, l, pt);
      size_t gi; int i, j, k;
      if (map.at(l, pt, gi, i, j, k)) {
        T q = X[l * ldx + pt] * K[gi];
        if (Cj) q += Cj[gi] * u[gi];
        X[l * ldx + pt] = q;
      }
    }
    __syncthreads();
    if (threadIdx.x < TL) {
      ends[2 * TL + threadIdx.x * 2 + 0] = X[threadIdx.x * ldx + 0];
      ends[2 * TL + threadIdx.x * 2 + 1] = X[threadIdx.x * ldx + N];
    }
    tile_deriv<T, ROUTE, P, CM, false, TL>(X, tmp, ldx, Cb, tw, Dm, n, ax.scale, ch, bh);
    const bool first = (kind == kApplyFirst || kind == kJacFirst);
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
      int l, pt; map.split(e, n, l, pt);
      size_t gi; int i, j, k;
      if (!map.at(l, pt, gi, i, j, k)) continue;
      const int o = owner_face(g, i, j, k);
      if (o < 0) {
        const T v = -X[l * ldx + pt];
        if (first) out[gi] = v;
        else out[gi] += v;
      } else if (g.bc[o] == CHEB_DIRICHLET) {
        if (first) out[gi] = u[gi];
      } else if ((o >> 1) == axis) {
        // hi face (side 1) is line point 0, lo face (side 0) is point N
        if (g.bc[o] == CHEB_FLUX)
          out[gi] = (o & 1) ? -ends[2 * TL + l * 2 + 0] : ends[2 * TL + l * 2 + 1];
        else
          out[gi] = (o & 1) ? ends[l * 2 + 0] : -ends[l * 2 + 1];
      } else if (first) {
        out[gi] = (T)0;  // Neumann / flux row of a later axis: written by that pass
      }
    }
  } else {
    // ---- A^T lam for this axis: D_a^T (S_a lam - K * D_a^T (P_int lam))
    // S_a lam: +-lam at line ends owned by a Neumann face of this axis,
    // -+K lam at ends owned by a flux face.
    if (threadIdx.x < TL) {
      const int l = threadIdx.x;
      size_t gi; int i, j, k;
      T s0 = (T)0, sN = (T)0;
      if (map.at(l, 0, gi, i, j, k)) {
        const int o = owner_face(g, i, j, k);
        if (o == 2 * axis + 1 && g.bc[o] == CHEB_NEUMANN) s0 = X[l * ldx + 0];
        if (o == 2 * axis + 1 && g.bc[o] == CHEB_FLUX) s0 = -K[gi] * X[l * ldx + 0];
      }
      if (map.at(l, N, gi, i, j, k)) {
        const int o = owner_face(g, i, j, k);
        if (o == 2 * axis && g.bc[o] == CHEB_NEUMANN) sN = -X[l * ldx + N];
        if (o == 2 * axis && g.bc[o] == CHEB_FLUX) sN = K[gi] * X[l * ldx + N];
      }
      ends[l * 2 + 0] = s0;
      ends[l * 2 + 1] = sN;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
      int l, pt; map.split(e, n, l, pt);
      size_t gi; int i, j, k;
      if (map.at(l, pt, gi, i, j, k) && owner_face(g, i, j, k) >= 0) X[l * ldx + pt] = (T)0;
    }
    tile_deriv<T, ROUTE, P, CM, true, TL>(X, tmp, ldx, Cb, tw, Dm, n, ax.scale, ch, bh);
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
      int l, pt; map.split(e, n, l, pt);
      size_t gi; int i, j, k;
      T v = (T)0;
      if (map.at(l, pt, gi, i, j, k)) {
        v = -K[gi] * X[l * ldx + pt];
        if (pt == 0) v += ends[l * 2 + 0];
        if (pt == N) v += ends[l * 2 + 1];
      }
      X[l * ldx + pt] = v;
    }
    tile_deriv<T, ROUTE, P, CM, true, TL>(X, tmp, ldx, Cb, tw, Dm, n, ax.scale, ch, bh);
    const bool first = (kind == kAdjFirst);
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
      int l, pt; map.split(e, n, l, pt);
      size_t gi; int i, j, k;
      if (!map.at(l, pt, gi, i, j, k)) continue;
      T v = X[l * ldx + pt];
      if (first) {
        const int o = owner_face(g, i, j, k);
        if (o >= 0 && g.bc[o] == CHEB_DIRICHLET) v += u[gi];
        out[gi] = v;
      } else {
        out[gi] += v;
      }
    }
  }
}

template <typename T, int ROUTE, int P, int CM, int TL>
__global__ void __launch_bounds__(TL * 16)
line_pass_kernel(Geom g, int axis, int kind, AxisK<T> ax, const T* __restrict__ K,
                 const T* __restrict__ u, T* __restrict__ out, const T* __restrict__ Cj) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PassSmem<T> sm = pass_stage<T, ROUTE, P, TL>(smem_raw, ax);
  line_pass_tile<T, ROUTE, P, CM, TL>(g, axis, kind, ax, K, u, out, Cj, blockIdx.x, sm);
}

}  // namespace cheb
