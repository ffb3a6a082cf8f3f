// Device building blocks of the line passes: complex arithmetic, the
// boundary-node owner rule, a warp-synchronous Stockham FFT, and the
// parity-interleaved scans that implement the Chebyshev derivative
// recurrence and its transpose.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace cheb {

template <typename T> struct C2;
template <> struct C2<float> { typedef float2 t; };
template <> struct C2<double> { typedef double2 t; };

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// multiply by -i
template <typename C>
__device__ __forceinline__ C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

// Owner face of node (i, j, k), or -1 for interior nodes.  Dirichlet faces
// beat Neumann faces; among faces of one type the lowest axis wins.  Node
// index 0 of an axis is its hi face (side 1), index n-1 its lo face.
__device__ __forceinline__ int owner_face(const Geom& g, int i, int j, int k) {
  int best_d = -1, best_n = -1;
  const int idx[3] = {i, j, k};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.dim) break;
    int f = -1;
    if (idx[a] == 0) f = 2 * a + 1;
    else if (idx[a] == g.n[a] - 1) f = 2 * a;
    if (f >= 0) {
      if (g.bc[f] == CHEB_DIRICHLET) { if (best_d < 0) best_d = f; }
      else { if (best_n < 0) best_n = f; }
    }
  }
  return best_d >= 0 ? best_d : best_n;
}

// ---------------------------------------------------------------------------
// Radix-R forward DFT butterflies (sign -1), in registers.
// ---------------------------------------------------------------------------
template <typename T, int R> struct Dft;

template <typename T> struct Dft<T, 2> {
  typedef typename C2<T>::t C;
  __device__ __forceinline__ static void run(C* v) {
    C a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};

template <typename T> struct Dft<T, 4> {
  typedef typename C2<T>::t C;
  __device__ __forceinline__ static void run(C* v) {
    C b0 = cadd(v[0], v[2]), b2 = csub(v[0], v[2]);
    C b1 = cadd(v[1], v[3]), b3 = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(b0, b1);
    v[2] = csub(b0, b1);
    v[1] = cadd(b2, b3);
    v[3] = csub(b2, b3);
  }
};

template <typename T> struct Dft<T, 8> {
  typedef typename C2<T>::t C;
  __device__ __forceinline__ static void run(C* v) {
    const T h = (T)0.70710678118654752440;
    // decimation in frequency: first distance-4 butterflies with w8^n twiddles
    C a0 = cadd(v[0], v[4]), a4 = csub(v[0], v[4]);
    C a1 = cadd(v[1], v[5]), a5 = csub(v[1], v[5]);
    C a2 = cadd(v[2], v[6]), a6 = csub(v[2], v[6]);
    C a3 = cadd(v[3], v[7]), a7 = csub(v[3], v[7]);
    // a5 w8 = h p5 (w8 = h (1 - i)), a7 w8^3 = h p7 (w8^3 = h (-1 - i)), a6 w8^2 = -i a6;
    // the factor h is applied by the output FMAs
    C p5, p7;
    p5.x = a5.x + a5.y; p5.y = a5.y - a5.x;
    p7.x = a7.y - a7.x; p7.y = -(a7.x + a7.y);
    a6 = cmul_mi(a6);
    C b0 = cadd(a0, a2), b2 = csub(a0, a2);
    C b1 = cadd(a1, a3), b3 = cmul_mi(csub(a1, a3));
    C b4 = cadd(a4, a6), b6 = csub(a4, a6);
    const C q5 = cadd(p5, p7), q7 = cmul_mi(csub(p5, p7));  // b5 = h q5, b7 = h q7
    v[0] = cadd(b0, b1);
    v[4] = csub(b0, b1);
    v[2] = cadd(b2, b3);
    v[6] = csub(b2, b3);
    v[1].x = b4.x + h * q5.x; v[1].y = b4.y + h * q5.y;
    v[5].x = b4.x - h * q5.x; v[5].y = b4.y - h * q5.y;
    v[3].x = b6.x + h * q7.x; v[3].y = b6.y + h * q7.y;
    v[7].x = b6.x - h * q7.x; v[7].y = b6.y - h * q7.y;
  }
};

// Padded position of element idx of a warp FFT buffer: one spare slot every
// 8 complex values keeps the strided Stockham stores free of bank conflicts.
__host__ __device__ __forceinline__ int fpad(int idx) { return idx + (idx >> 3); }
template <int P> struct FftBuf { static constexpr int len = P + P / 8; };

// One Stockham stage of radix R on a length-P sequence held in shared
// memory by one warp (in place: every lane reads its butterflies into
// registers, the warp synchronises, then every lane writes).  Ns is the
// product of the radices of the earlier stages.  Stage twiddles are stored
// contiguously: tw[(Ns - 1) + (r - 1) Ns + k] = exp(-2 pi i r k / (Ns R)).
template <typename T, int P, int R, int Ns>
__device__ __forceinline__ void warp_stage(typename C2<T>::t* buf, const typename C2<T>::t* tw,
                                           int lane) {
  typedef typename C2<T>::t C;
  constexpr int NB = P / R;                 // butterflies
  constexpr int IT = (NB + 31) / 32;        // butterflies per lane
  C v[IT][R];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = lane + 32 * it;
    if (NB % 32 == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[it][r] = buf[fpad(j + r * NB)];
      if (Ns > 1) {
        const int k = j & (Ns - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) v[it][r] = cmul(v[it][r], tw[(Ns - 1) + (r - 1) * Ns + k]);
      }
      Dft<T, R>::run(v[it]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = lane + 32 * it;
    if (NB % 32 == 0 || j < NB) {
      const int k = j & (Ns - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[fpad(base + r * Ns)] = v[it][r];
    }
  }
  __syncwarp();
}

// Stage sequence: radix 8 while possible, then one radix-4 or radix-2 stage.
template <typename T, int P, int Ns, int REM>
struct WarpFft {
  __device__ __forceinline__ static void run(typename C2<T>::t* buf, const typename C2<T>::t* tw,
                                             int lane) {
    if constexpr (REM >= 8 && REM % 8 == 0) {
      warp_stage<T, P, 8, Ns>(buf, tw, lane);
      WarpFft<T, P, Ns * 8, REM / 8>::run(buf, tw, lane);
    } else if constexpr (REM == 4) {
      warp_stage<T, P, 4, Ns>(buf, tw, lane);
    } else if constexpr (REM == 2) {
      warp_stage<T, P, 2, Ns>(buf, tw, lane);
    }
  }
};

// Forward DFT of length P (power of two, 8..1024) of buf (padded layout).
template <typename T, int P>
__device__ __forceinline__ void warp_fft(typename C2<T>::t* buf, const typename C2<T>::t* tw,
                                         int lane) {
  WarpFft<T, P, 1, P>::run(buf, tw, lane);
}

// ---------------------------------------------------------------------------
// DFT of any length M by Bluestein's chirp-z identity (L. I. Bluestein, "A
// linear filtering approach to the computation of the discrete Fourier
// transform", 1970).  With c_j = exp(-i pi j^2 / M), jk = (j^2 + k^2 -
// (k - j)^2) / 2 gives
//   X_k = sum_{j<M} x_j exp(-2 pi i jk / M) = c_k sum_{j<M} (x_j c_j) conj(c_{k-j}),
// a circular convolution of length L (a power of two, L >= 2M - 1, so the
// wrapped kernel b_m = conj(c_|m|), |m| < M, does not alias).  It is
// evaluated with two length-L warp FFTs: FFT(conj(A * B)) = L conj(IFFT(A * B)).
// bhat = FFT_L(b) / L is a plan table; chirp holds c_j for j < M.
// On entry buf[fpad(j)] holds x_j for j < M (later entries are ignored); on
// exit buf[fpad(k)] holds X_k for k < M.
// ---------------------------------------------------------------------------
template <typename T, int L>
__device__ __noinline__ void warp_dft_chirp(typename C2<T>::t* buf, const typename C2<T>::t* tw,
                                               const typename C2<T>::t* chirp,
                                               const typename C2<T>::t* bhat, int M, int lane) {
  typedef typename C2<T>::t C;
  for (int j = lane; j < L; j += 32) {
    C v;
    if (j < M) {
      v = cmul(buf[fpad(j)], chirp[j]);
    } else {
      v.x = (T)0;
      v.y = (T)0;
    }
    buf[fpad(j)] = v;
  }
  __syncwarp();
  warp_fft<T, L>(buf, tw, lane);
  for (int k = lane; k < L; k += 32) {
    C v = cmul(buf[fpad(k)], bhat[k]);
    v.y = -v.y;
    buf[fpad(k)] = v;
  }
  __syncwarp();
  warp_fft<T, L>(buf, tw, lane);
  for (int k = lane; k < M; k += 32) {
    C v = buf[fpad(k)];
    v.y = -v.y;
    buf[fpad(k)] = cmul(chirp[k], v);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Parity-interleaved scans on one line x[0..N] held in shared memory, by one
// warp.  SUFFIX: x_k <- sum_{j > k, j - k odd} x_j for k < N, x_N <- 0
// (the backward derivative recurrence in closed form).  PREFIX (its
// transpose): x_j <- sum_{k < j, j - k odd} x_k for j >= 1, x_0 <- 0.
// Each parity class is split into contiguous lane chunks; lane totals are
// combined with shuffles.  CM = max elements per lane per class.
// ---------------------------------------------------------------------------
template <typename T, int CM, bool SUFFIX>
__device__ __forceinline__ void warp_parity_scan(T* x, int N, int lane) {
  T val[2][CM];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int t = 0; t < CM; ++t) val[q][t] = (T)0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int M = (N - q) / 2 + 1;  // elements q, q+2, ... <= N
    const int c = (M + 31) / 32;
    const int i0 = lane * c;
    T tot = 0;
    if (SUFFIX) {
#pragma unroll
      for (int t = CM - 1; t >= 0; --t) {
        const int i = i0 + t;
        if (t < c && i < M) { tot += x[q + 2 * i]; val[q][t] = tot; }
      }
      // inclusive suffix of lane totals, then shift by one lane (exclusive)
      T acc = tot;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_down_sync(0xffffffffu, acc, d);
        if (lane + d < 32) acc += o;
      }
      T excl = __shfl_down_sync(0xffffffffu, acc, 1);
      if (lane == 31) excl = (T)0;
#pragma unroll
      for (int t = 0; t < CM; ++t) val[q][t] += excl;
    } else {
#pragma unroll
      for (int t = 0; t < CM; ++t) {
        const int i = i0 + t;
        if (t < c && i < M) { tot += x[q + 2 * i]; val[q][t] = tot; }
      }
      T acc = tot;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, acc, d);
        if (lane >= d) acc += o;
      }
      T excl = __shfl_up_sync(0xffffffffu, acc, 1);
      if (lane == 0) excl = (T)0;
#pragma unroll
      for (int t = 0; t < CM; ++t) val[q][t] += excl;
    }
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int M = (N - q) / 2 + 1;
    const int c = (M + 31) / 32;
    const int i0 = lane * c;
#pragma unroll
    for (int t = 0; t < CM; ++t) {
      const int i = i0 + t;
      if (t < c && i < M) {
        const int m = q + 2 * i;  // inclusive scan value sits at m
        if (SUFFIX) { if (m >= 1) x[m - 1] = val[q][t]; }
        else { if (m + 1 <= N) x[m + 1] = val[q][t]; }
      }
    }
  }
  if (lane == 0) {
    if (SUFFIX) x[N] = (T)0;
    else x[0] = (T)0;
  }
  __syncwarp();
}

}  // namespace cheb
