// Line passes of the collocation operator (Alg. 1 and Alg. 3 of the paper,
// Sec. 2.2 / Sec. 2.3.2) and the right-hand side with boundary rows.
//
// One CTA owns a tile of TL lines along one axis (TL = 8 or 16, chosen per
// axis and precision by the plan's autotuner; 16 TL threads, two lines per
// warp).  The tile is staged in shared memory with coalesced loads: for the
// x axis the lines are contiguous in memory, for y and z the tile holds TL
// x-adjacent lines so every row of the tile is a contiguous run of TL elements.
//
// Line derivative, transform route (N = n - 1, P = 2N a power of two):
//   F = DCT-I(f) as the real part of a length-P FFT of the even extension
//       (two lines share one complex FFT: line A real part, line B imaginary),
//   G_k = k c_k (2/(hi-lo)) F_k / N      (c_N = 1/2: a_k = c_k F_k / N),
//   beta_k = sum_{j>k, j-k odd} G_j      (the backward recurrence
//       b_{k-1} = b_{k+1} + 2k a_k with b_0 halved, in closed form, as a
//       parity-interleaved warp suffix scan; beta_k = b_k / 2, beta_N = 0),
//   f' = DCT-I(beta)                      (= sum_k b_k T_k at the nodes).
// Each line pair is processed by one warp without block-wide barriers.
// Dense route: f' = D f with D staged in shared memory.
#include <cstdio>

#include "line_pass.cuh"
#include "umma.h"

namespace cheb {

// ---------------------------------------------------------------------------
// transform-route pass with compile-time N: tiles staged by cp.async (u, then
// K, then the accumulated output) so the loads overlap the warp FFTs
// ---------------------------------------------------------------------------
template <int B>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (B == 4) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NW>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NW) : "memory"); }

template <typename T, int P, int TL>
__host__ __device__ constexpr size_t tf_smem_bytes() {
  return align16(sizeof(T) * TL * (P / 2 + 1)) * 2 + align16(sizeof(T) * TL * 4) +
         align16(2 * sizeof(T) * (size_t)(TL / 2) * FftBuf<P>::len) + align16(2 * sizeof(T) * (size_t)P);
}

template <typename T, int P, int CM, int TL>
__global__ void __launch_bounds__(TL * 16, 2)
tf_pass_kernel(Geom g, int axis, int kind, AxisK<T> ax, const T* __restrict__ K,
               const T* __restrict__ u, T* __restrict__ out, const T* __restrict__ Cj) {
  typedef typename C2<T>::t C;
  constexpr int N = P / 2, n = N + 1, ldx = n;  // n is odd
  constexpr int NT = TL * 16;                     // threads: two lines per warp
  constexpr int TE = TL * n;
  constexpr int BL = FftBuf<P>::len;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* p = smem_raw;
  T* X = (T*)p;    p += align16(sizeof(T) * TL * ldx);
  T* KO = (T*)p;   p += align16(sizeof(T) * TL * ldx);
  T* ends = (T*)p; p += align16(sizeof(T) * TL * 4);
  C* Cb = (C*)p;   p += align16(2 * sizeof(T) * (size_t)(TL / 2) * BL);
  C* tw = (C*)p;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const bool adj = (kind == kAdjFirst || kind == kAdjAcc);
  const bool is_acc = (kind == kApplyAcc || kind == kAdjAcc || kind == kJacAcc);
  const bool first = (kind == kApplyFirst || kind == kAdjFirst || kind == kJacFirst);
  const bool needK = !(kind == kDeriv || kind == kDerivT);
  // tile geometry
  int line0 = 0, i0 = 0, outer = 0;
  size_t base = 0, pstride = 1;
  if (axis == 0) {
    line0 = blockIdx.x * TL;
  } else {
    const int nbx = (nx + TL - 1) / TL;
    i0 = (blockIdx.x % nbx) * TL;
    outer = blockIdx.x / nbx;
    if (axis == 1) { base = (size_t)outer * ny * nx + i0; pstride = nx; }
    else { base = (size_t)outer * nx + i0; pstride = (size_t)nx * ny; }
  }
  const int nlines = ny * nz;
  auto elem = [&](int e, int& l, int& pt, size_t& gi) -> bool {
    if (axis == 0) {
      l = e / n;
      pt = e - l * n;
      gi = (size_t)line0 * n + e;
      return line0 + l < nlines;
    }
    l = e % TL;
    pt = e / TL;
    gi = base + (size_t)pt * pstride + l;
    return i0 + l < nx;
  };
  auto node = [&](int l, int pt, int& i, int& j, int& k) {
    if (axis == 0) { const int line = line0 + l; i = pt; j = line % ny; k = line / ny; }
    else if (axis == 1) { i = i0 + l; j = pt; k = outer; }
    else { i = i0 + l; j = outer; k = pt; }
  };
  auto gindex = [&](int l, int pt) -> size_t {  // global index of tile element (l, pt)
    if (axis == 0) return (size_t)(line0 + l) * n + pt;
    return base + (size_t)pt * pstride + l;
  };
  auto on_bnd = [&](int i, int j, int k) -> bool {
    bool b = (i == 0 || i == nx - 1);
    if (g.dim > 1) b = b || j == 0 || j == ny - 1;
    if (g.dim > 2) b = b || k == 0 || k == nz - 1;
    return b;
  };
  // ---- stage twiddles and launch the tile copies
  for (int t = threadIdx.x; t < P; t += NT) tw[t] = ax.tw[t];
  for (int e = threadIdx.x; e < TE; e += NT) {
    int l, pt; size_t gi;
    if (elem(e, l, pt, gi)) cp_async<sizeof(T)>(&X[l * ldx + pt], u + gi);
    else X[l * ldx + pt] = (T)0;
  }
  cp_commit();
  if (needK) {
    for (int e = threadIdx.x; e < TE; e += NT) {
      int l, pt; size_t gi;
      if (elem(e, l, pt, gi)) cp_async<sizeof(T)>(&KO[l * ldx + pt], K + gi);
      else KO[l * ldx + pt] = (T)0;
    }
  }
  cp_commit();
  cp_wait<1>();
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  C* buf = Cb + (size_t)w * BL;

  if (kind == kDeriv || kind == kDerivT) {
    if (kind == kDeriv) warp_deriv_tf<T, P, CM, false>(X, ldx, buf, tw, N, ax.scale, w, lane);
    else warp_deriv_tf<T, P, CM, true>(X, ldx, buf, tw, N, ax.scale, w, lane);
    __syncthreads();
    for (int e = threadIdx.x; e < TE; e += NT) {
      int l, pt; size_t gi;
      if (elem(e, l, pt, gi)) out[gi] = X[l * ldx + pt];
    }
    return;
  }

  if (!adj) {
    warp_deriv_tf<T, P, CM, false>(X, ldx, buf, tw, N, ax.scale, w, lane);
    __syncthreads();
    if (threadIdx.x < TL) {
      ends[threadIdx.x * 2 + 0] = X[threadIdx.x * ldx + 0];
      ends[threadIdx.x * 2 + 1] = X[threadIdx.x * ldx + N];
    }
    cp_wait<0>();
    __syncthreads();
    if (Cj) {
      // Jacobian action: q = K D_a du + C_a du (coalesced reads of C_a and du)
      for (int e = threadIdx.x; e < TE; e += NT) {
        int l, pt; size_t gi;
        const bool in = elem(e, l, pt, gi);
        T q = X[l * ldx + pt] * KO[l * ldx + pt];
        if (in) q += Cj[gi] * u[gi];
        X[l * ldx + pt] = q;
      }
    } else {
      for (int e = threadIdx.x; e < TE; e += NT) {
        const int l = e / n, pt = e - (e / n) * n;
        X[l * ldx + pt] *= KO[l * ldx + pt];
      }
    }
    __syncthreads();
    if (threadIdx.x < TL) {  // line ends of K D_a u for flux rows
      ends[2 * TL + threadIdx.x * 2 + 0] = X[threadIdx.x * ldx + 0];
      ends[2 * TL + threadIdx.x * 2 + 1] = X[threadIdx.x * ldx + N];
    }
    __syncthreads();
    if (is_acc) {  // prefetch the output being accumulated into the free K tile
      for (int e = threadIdx.x; e < TE; e += NT) {
        int l, pt; size_t gi;
        if (elem(e, l, pt, gi)) cp_async<sizeof(T)>(&KO[l * ldx + pt], out + gi);
      }
      cp_commit();
    }
    warp_deriv_tf<T, P, CM, false>(X, ldx, buf, tw, N, ax.scale, w, lane);
    cp_wait<0>();
    __syncthreads();
    for (int e = threadIdx.x; e < TE; e += NT) {
      int l, pt; size_t gi;
      if (!elem(e, l, pt, gi)) continue;
      int i, j, k;
      node(l, pt, i, j, k);
      const T v = -X[l * ldx + pt];
      if (!on_bnd(i, j, k)) {
        out[gi] = first ? v : KO[l * ldx + pt] + v;
        continue;
      }
      const int o = owner_face(g, i, j, k);
      if (g.bc[o] == CHEB_DIRICHLET) {
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
    return;
  }

  // ---- A^T lam for this axis: D_a^T (S_a lam - K * D_a^T (P_int lam))
  if (threadIdx.x < TL) {
    const int l = threadIdx.x;
    T s0 = (T)0, sN = (T)0;
    int e0l, e0p; size_t gi;
    if (elem(l * (axis == 0 ? n : 1), e0l, e0p, gi)) {
      int i, j, k;
      node(l, 0, i, j, k);
      const int o = owner_face(g, i, j, k);
      if (o == 2 * axis + 1 && g.bc[o] == CHEB_NEUMANN) s0 = X[l * ldx + 0];
      if (o == 2 * axis + 1 && g.bc[o] == CHEB_FLUX) s0 = -K[gindex(l, 0)] * X[l * ldx + 0];
      node(l, N, i, j, k);
      const int o2 = owner_face(g, i, j, k);
      if (o2 == 2 * axis && g.bc[o2] == CHEB_NEUMANN) sN = -X[l * ldx + N];
      if (o2 == 2 * axis && g.bc[o2] == CHEB_FLUX) sN = K[gindex(l, N)] * X[l * ldx + N];
    }
    ends[l * 2 + 0] = s0;
    ends[l * 2 + 1] = sN;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TE; e += NT) {
    int l, pt; size_t gi;
    if (!elem(e, l, pt, gi)) continue;
    int i, j, k;
    node(l, pt, i, j, k);
    if (on_bnd(i, j, k)) X[l * ldx + pt] = (T)0;
  }
  __syncthreads();
  warp_deriv_tf<T, P, CM, true>(X, ldx, buf, tw, N, ax.scale, w, lane);
  cp_wait<0>();
  __syncthreads();
  for (int e = threadIdx.x; e < TE; e += NT) {
    const int l = e / n, pt = e - (e / n) * n;
    T v = -KO[l * ldx + pt] * X[l * ldx + pt];
    if (pt == 0) v += ends[l * 2 + 0];
    if (pt == N) v += ends[l * 2 + 1];
    X[l * ldx + pt] = v;
  }
  __syncthreads();
  if (is_acc) {
    for (int e = threadIdx.x; e < TE; e += NT) {
      int l, pt; size_t gi;
      if (elem(e, l, pt, gi)) cp_async<sizeof(T)>(&KO[l * ldx + pt], out + gi);
    }
    cp_commit();
  }
  warp_deriv_tf<T, P, CM, true>(X, ldx, buf, tw, N, ax.scale, w, lane);
  cp_wait<0>();
  __syncthreads();
  for (int e = threadIdx.x; e < TE; e += NT) {
    int l, pt; size_t gi;
    if (!elem(e, l, pt, gi)) continue;
    T v = X[l * ldx + pt];
    if (first) {
      int i, j, k;
      node(l, pt, i, j, k);
      if (on_bnd(i, j, k)) {
        const int o = owner_face(g, i, j, k);
        if (g.bc[o] == CHEB_DIRICHLET) v += u[gi];
      }
      out[gi] = v;
    } else {
      out[gi] = KO[l * ldx + pt] + v;
    }
  }
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
template <typename T> static AxisK<T> axis_k(const AxisTables& t);
template <> AxisK<double> axis_k<double>(const AxisTables& t) {
  AxisK<double> a;
  a.n = t.n; a.N = t.N; a.scale = t.scale; a.tw = t.tw64; a.chirp = t.chirp64; a.bhat = t.bhat64; a.D = t.D64;
  return a;
}
template <> AxisK<float> axis_k<float>(const AxisTables& t) {
  AxisK<float> a;
  a.n = t.n; a.N = t.N; a.scale = (float)t.scale; a.tw = t.tw32; a.chirp = t.chirp32; a.bhat = t.bhat32;
  a.D = t.D32;
  return a;
}

template <typename T, int ROUTE, int P, int CM, int TL>
static int launch_kernel(const Geom& g, int axis, int kind, const AxisK<T>& ak, const T* K,
                         const T* u, T* out, cudaStream_t s, int nblocks, const T* C) {
  int st;
  if constexpr (ROUTE == CHEB_ROUTE_TRANSFORM) {
    auto kern = tf_pass_kernel<T, P, CM, TL>;
    constexpr size_t smem = tf_smem_bytes<T, P, TL>();
    if ((st = ensure_smem_attr((const void*)kern, smem))) return st;
    kern<<<nblocks, TL * 16, smem, s>>>(g, axis, kind, ak, K, u, out, C);
    CHEB_LAUNCH_CHECK("tf_pass_kernel");
  } else {
    auto kern = line_pass_kernel<T, ROUTE, P, CM, TL>;
    const size_t smem = pass_smem_bytes<T>(ROUTE, ak.n, P, TL);
    if ((st = ensure_smem_attr((const void*)kern, smem))) return st;
    kern<<<nblocks, TL * 16, smem, s>>>(g, axis, kind, ak, K, u, out, C);
    CHEB_LAUNCH_CHECK("line_pass_kernel");
  }
  return CHEB_OK;
}

template <typename T, int TL>
static int dispatch_pass(const cheb_plan_s* p, int axis, int kind, int route, const T* K, const T* u, T* out,
                         cudaStream_t s, const T* C) {
  const Geom g = p->geom();
  const AxisTables& t = p->ax[axis];
  const AxisK<T> ak = axis_k<T>(t);
  int nblocks;
  if (axis == 0) nblocks = (g.n[1] * g.n[2] + TL - 1) / TL;
  else {
    const int nbx = (g.n[0] + TL - 1) / TL;
    nblocks = nbx * (axis == 1 ? g.n[2] : g.n[1]);
  }
  if (nblocks == 0) return CHEB_OK;
  if (route == CHEB_ROUTE_DENSE)
    return launch_kernel<T, CHEB_ROUTE_DENSE, 0, 1, TL>(g, axis, kind, ak, K, u, out, s, nblocks, C);
  if (t.chirp) return launch_chirp_pass<T>(g, axis, kind, ak, t.P, K, u, out, s, C);
  switch (t.P) {
    case 8: return launch_kernel<T, CHEB_ROUTE_TRANSFORM, 8, 1, TL>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 16: return launch_kernel<T, CHEB_ROUTE_TRANSFORM, 16, 1, TL>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 32: return launch_kernel<T, CHEB_ROUTE_TRANSFORM, 32, 1, TL>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 64: return launch_kernel<T, CHEB_ROUTE_TRANSFORM, 64, 1, TL>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 128: return launch_kernel<T, CHEB_ROUTE_TRANSFORM, 128, 2, TL>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 256: return launch_kernel<T, CHEB_ROUTE_TRANSFORM, 256, 3, TL>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 512: return launch_kernel<T, CHEB_ROUTE_TRANSFORM, 512, 5, TL>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    default:
      set_error("transform route needs 2N a power of two in [8, 512]");
      return CHEB_ERR_UNSUPPORTED;
  }
}

template <typename T>
int launch_pass(const cheb_plan_s* p, int axis, int kind, const T* K, const T* u, T* out,
                cudaStream_t s, const T* C) {
  const AxisTables& t = p->ax[axis];
  int route = sizeof(T) == 4 ? t.route32 : t.route;
  if (route == CHEB_ROUTE_TENSOR) {
    if constexpr (sizeof(T) == 4) {
      if (kind == kApplyFirst || kind == kApplyAcc)
        return tensor_apply_pass(p, axis, kind == kApplyFirst, K, u, out, s);
    }
    route = line_route(t);
  }
  const int tile = sizeof(T) == 4 ? t.tile32 : t.tile;
  if (tile == 8) return dispatch_pass<T, 8>(p, axis, kind, route, K, u, out, s, C);
  return dispatch_pass<T, 16>(p, axis, kind, route, K, u, out, s, C);
}

template int launch_pass<double>(const cheb_plan_s*, int, int, const double*, const double*, double*, cudaStream_t,
                                 const double*);
template int launch_pass<float>(const cheb_plan_s*, int, int, const float*, const float*, float*, cudaStream_t,
                                const float*);

template <typename T>
int launch_apply(const cheb_plan_s* p, const T* K, const T* u, T* out, cudaStream_t s) {
  for (int a = 0; a < p->dim; ++a) {
    int st = launch_pass<T>(p, a, a == 0 ? kApplyFirst : kApplyAcc, K, u, out, s);
    if (st != CHEB_OK) return st;
  }
  return CHEB_OK;
}
template int launch_apply<double>(const cheb_plan_s*, const double*, const double*, double*, cudaStream_t);
template int launch_apply<float>(const cheb_plan_s*, const float*, const float*, float*, cudaStream_t);

template <typename T>
int launch_jacobian(const cheb_plan_s* p, const T* K, const T* const C[3], const T* du, T* out, cudaStream_t s) {
  for (int a = 0; a < p->dim; ++a) {
    int st = launch_pass<T>(p, a, a == 0 ? kJacFirst : kJacAcc, K, du, out, s, C[a]);
    if (st != CHEB_OK) return st;
  }
  return CHEB_OK;
}
template int launch_jacobian<double>(const cheb_plan_s*, const double*, const double* const*, const double*, double*,
                                     cudaStream_t);
template int launch_jacobian<float>(const cheb_plan_s*, const float*, const float* const*, const float*, float*,
                                    cudaStream_t);

template <typename T>
int launch_adjoint_apply(const cheb_plan_s* p, const T* K, const T* lam, T* out, cudaStream_t s) {
  for (int a = 0; a < p->dim; ++a) {
    int st = launch_pass<T>(p, a, a == 0 ? kAdjFirst : kAdjAcc, K, lam, out, s);
    if (st != CHEB_OK) return st;
  }
  return CHEB_OK;
}
template int launch_adjoint_apply<double>(const cheb_plan_s*, const double*, const double*, double*, cudaStream_t);
template int launch_adjoint_apply<float>(const cheb_plan_s*, const float*, const float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// right-hand side with boundary rows
// ---------------------------------------------------------------------------
struct FacePtrs { const double* f[6]; };

__global__ void rhs_kernel(Geom g, const double* f, FacePtrs faces, double* b) {
  const size_t total = (size_t)g.n[0] * g.n[1] * g.n[2];
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.n[0]);
    const int j = (int)((idx / g.n[0]) % g.n[1]);
    const int k = (int)(idx / ((size_t)g.n[0] * g.n[1]));
    const int o = owner_face(g, i, j, k);
    if (o < 0) { b[idx] = f[idx]; continue; }
    const int a = o >> 1;
    size_t fi;
    if (a == 0) fi = (size_t)k * g.n[1] + j;
    else if (a == 1) fi = (size_t)k * g.n[0] + i;
    else fi = (size_t)j * g.n[0] + i;
    b[idx] = faces.f[o][fi];
  }
}

int launch_rhs(const cheb_plan_s* p, const double* f, const double* const face_vals[6], double* b,
               cudaStream_t s) {
  FacePtrs fp;
  for (int i = 0; i < 6; ++i) fp.f[i] = face_vals[i];
  const size_t total = p->size();
  int blocks = (int)std::min<size_t>((total + 255) / 256, 148 * 16);
  rhs_kernel<<<blocks, 256, 0, s>>>(p->geom(), f, fp, b);
  CHEB_LAUNCH_CHECK("rhs_kernel");
  return CHEB_OK;
}

}  // namespace cheb
