// Lockstep batched solves: many independent grids (different sizes and
// boundary sets) iterate together.  The data path of one Arnoldi step of
// every active instance is a handful of launches, captured as one CUDA graph
// and replayed per step:
//   * the operator apply: per axis, one persistent grid over the work list
//     of (instance, line tile) items of all instances (the generic line
//     pass, dense route, line_pass.cuh), so small grids share the GPU;
//   * the preconditioner: each instance's fast-diagonalisation inverse as a
//     parallel branch of the graph;
//   * the Gram-Schmidt multi-dot and multi-axpy over the concatenated
//     vectors, with per-instance coefficients and deterministic
//     per-instance reductions;
//   * the Hessenberg column and Givens rotation of every instance, one CTA
//     each; an instance whose residual estimate meets its tolerance clears
//     its bit in the device-side active mask, and every later kernel of the
//     cycle skips it.
// The refinement loop (FP32 inner LGMRES, FP64 residual) and the Picard
// loop run in lockstep on top, each instance leaving as it converges.
// Vectors of the batch are one allocation: instance i occupies elements
// [off_i, off_i + n_i), off_i a multiple of kBAlign.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fdm.h"
#include "hess.cuh"
#include "krylov.h"
#include "line_pass.cuh"

namespace cheb {

// plan-level helpers (solve.cu)
int plan_fdm(cheb_plan_s* p, Fdm** f);
int plan_kref(cheb_plan_s* p, const double* K, double* kref, cudaStream_t s);
void resolve_opts(const cheb_solve_opts* in, cheb_solve_opts* out);
bool pmat_ok(const cheb_solve_opts& o);

namespace {

constexpr int kBThreads = 256;
constexpr long long kBChunk = 8192;  // elements per vector-kernel block
constexpr long long kBAlign = 64;    // instance offsets (elements)
constexpr int kBTile = 16;           // lines per line-pass tile
constexpr int kDv = kMaxVecs + 2;    // per-instance device scalars: dots, |w|^2 (at kMaxVecs + 1)

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// vector kernels over the concatenated vectors
// ---------------------------------------------------------------------------
struct BatchBlocks {
  const int* inst;       // block -> instance
  const long long* lo;   // block element range [lo, hi)
  const long long* hi;
  const int* first;      // instance -> first block (ninst + 1 entries)
  int nblk, ninst;
};

template <typename T> struct BV;
template <> struct BV<float> { typedef float4 t; static constexpr int W = 4; };
template <> struct BV<double> { typedef double2 t; static constexpr int W = 2; };

template <typename T>
__device__ __forceinline__ T bget(const typename BV<T>::t& v, int k) {
  if constexpr (BV<T>::W == 4) return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
  else return k == 0 ? v.x : v.y;
}
template <typename T>
__device__ __forceinline__ void bset(typename BV<T>::t& v, int k, T x) {
  if constexpr (BV<T>::W == 4) {
    if (k == 0) v.x = x; else if (k == 1) v.y = x; else if (k == 2) v.z = x; else v.w = x;
  } else {
    if (k == 0) v.x = x; else v.y = x;
  }
}

// Block-reduce acc: slot l < cnt is output l and, when extra, slot MAXV-1
// is output cnt.  The block's sums go to part[o * nblk + block]; the last
// block to finish sums each instance's partials in block order (one warp
// per (instance, output) pair) into out[i * ostride + o].
template <int MAXV, typename T>
__device__ void bred_store(const BatchBlocks& bb, T (&acc)[MAXV], int cnt, bool extra, double* part,
                           unsigned* counter, double* out, int ostride) {
  __shared__ double sred[kBThreads / 32][MAXV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nout = cnt + (extra ? 1 : 0);
#pragma unroll
  for (int l = 0; l < MAXV; ++l) {
    const bool on = l < cnt || (extra && l == MAXV - 1);
    if (on) {
      const int o = l < cnt ? l : cnt;
      T v = acc[l];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
      if (lane == 0) sred[wid][o] = (double)v;
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kBThreads / 32; ++w) s += sred[w][o];
    part[(size_t)o * bb.nblk + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)(gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int q = wid; q < bb.ninst * nout; q += kBThreads / 32) {
    const int i = q / nout, o = q - i * nout;
    double s = 0.0;
    for (int b = bb.first[i] + lane; b < bb.first[i + 1]; b += 32) s += __ldcg(part + (size_t)o * bb.nblk + b);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) out[(size_t)i * ostride + o] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// 16-byte elements per thread and loop iteration: at least four independent
// loads in flight.  Resident CTAs asked of the register allocator: one from 16
// vectors on, where the loads in flight already cover the memory latency.
template <int NLOADS>
constexpr int bunroll() { return NLOADS >= 4 ? 1 : NLOADS >= 2 ? 2 : 4; }
template <int NV>
constexpr int bmin_ctas() { return NV >= 16 ? 1 : 2; }

// out[i][l] = <src_l, w> over instance i, l < NV; with_self: out[i][NV] = <w, w>.
// One instantiation per vector count NV, so no load or FMA of an absent
// vector is issued.
template <typename T, int NV>
__global__ void __launch_bounds__(kBThreads, bmin_ctas<NV>())
bmdot_kernel(BatchBlocks bb, VecList<T> src, const T* __restrict__ w, int with_self,
             const int* __restrict__ act, double* part, unsigned* counter, double* out) {
  typedef typename BV<T>::t V;
  constexpr int W = BV<T>::W;
  constexpr int U = bunroll<NV + 1>();
  T acc[NV + 1];
#pragma unroll
  for (int l = 0; l <= NV; ++l) acc[l] = (T)0;
  const int i = bb.inst[blockIdx.x];
  if (act[i]) {
    const long long lo = bb.lo[blockIdx.x], hi = bb.hi[blockIdx.x];
    const long long nv = (hi - lo) / W;
    const V* w4 = reinterpret_cast<const V*>(w + lo);
    long long e = threadIdx.x;
    for (; e + (U - 1) * (long long)blockDim.x < nv; e += U * (long long)blockDim.x) {
      V wv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) wv[u] = w4[e + u * blockDim.x];
#pragma unroll
      for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int l = 0; l < NV; ++l) {
          const V sv = reinterpret_cast<const V*>(src.p[l] + lo)[e + u * blockDim.x];
#pragma unroll
          for (int k = 0; k < W; ++k) acc[l] += bget<T>(sv, k) * bget<T>(wv[u], k);
        }
        if (with_self) {
#pragma unroll
          for (int k = 0; k < W; ++k) acc[NV] += bget<T>(wv[u], k) * bget<T>(wv[u], k);
        }
      }
    }
    for (; e < nv; e += blockDim.x) {
      const V wv = w4[e];
#pragma unroll
      for (int l = 0; l < NV; ++l) {
        const V sv = reinterpret_cast<const V*>(src.p[l] + lo)[e];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[l] += bget<T>(sv, k) * bget<T>(wv, k);
      }
      if (with_self) {
#pragma unroll
        for (int k = 0; k < W; ++k) acc[NV] += bget<T>(wv, k) * bget<T>(wv, k);
      }
    }
    for (long long t = lo + nv * W + threadIdx.x; t < hi; t += blockDim.x) {
      const T x = w[t];
#pragma unroll
      for (int l = 0; l < NV; ++l) acc[l] += src.p[l][t] * x;
      if (with_self) acc[NV] += x * x;
    }
  }
  bred_store<NV + 1, T>(bb, acc, NV, with_self != 0, part, counter, out, kDv);
}

// y_i = beta y_i + sum_l c_il src_l over instance i, l < NV (c_il = csign
// cdev[i kDv + l], or cmat[i * NV + l] when cdev is null); want_norm:
// |y_i|^2 -> norm[i kDv]
template <typename T, int NV>
__global__ void __launch_bounds__(kBThreads, bmin_ctas<NV>())
bmaxpy_kernel(BatchBlocks bb, VecList<T> src, const double* __restrict__ cdev, double csign,
              const double* __restrict__ cmat, double beta, T* __restrict__ y,
              const int* __restrict__ act, int want_norm, double* part, unsigned* counter, double* norm) {
  typedef typename BV<T>::t V;
  constexpr int W = BV<T>::W;
  constexpr int U = bunroll<NV + 1>();
  const int i = bb.inst[blockIdx.x];
  T acc[1] = {(T)0};
  if (act[i]) {
    T c[NV > 0 ? NV : 1];
#pragma unroll
    for (int l = 0; l < NV; ++l)
      c[l] = (T)(cdev ? csign * cdev[(size_t)i * kDv + l] : cmat[(size_t)i * NV + l]);
    const T b = (T)beta;
    const bool keep = beta != 0.0;
    const long long lo = bb.lo[blockIdx.x], hi = bb.hi[blockIdx.x];
    const long long nv = (hi - lo) / W;
    V* y4 = reinterpret_cast<V*>(y + lo);
    long long e = threadIdx.x;
    for (; e + (U - 1) * (long long)blockDim.x < nv; e += U * (long long)blockDim.x) {
      V v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (keep) {
          const V yo = y4[e + u * blockDim.x];
#pragma unroll
          for (int k = 0; k < W; ++k) bset<T>(v[u], k, b * bget<T>(yo, k));
        } else {
#pragma unroll
          for (int k = 0; k < W; ++k) bset<T>(v[u], k, (T)0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int l = 0; l < NV; ++l) {
          const V sv = reinterpret_cast<const V*>(src.p[l] + lo)[e + u * blockDim.x];
#pragma unroll
          for (int k = 0; k < W; ++k) bset<T>(v[u], k, bget<T>(v[u], k) + c[l] * bget<T>(sv, k));
        }
        y4[e + u * blockDim.x] = v[u];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[0] += bget<T>(v[u], k) * bget<T>(v[u], k);
      }
    }
    for (; e < nv; e += blockDim.x) {
      V v;
      if (keep) {
        const V yo = y4[e];
#pragma unroll
        for (int k = 0; k < W; ++k) bset<T>(v, k, b * bget<T>(yo, k));
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) bset<T>(v, k, (T)0);
      }
#pragma unroll
      for (int l = 0; l < NV; ++l) {
        const V sv = reinterpret_cast<const V*>(src.p[l] + lo)[e];
#pragma unroll
        for (int k = 0; k < W; ++k) bset<T>(v, k, bget<T>(v, k) + c[l] * bget<T>(sv, k));
      }
      y4[e] = v;
#pragma unroll
      for (int k = 0; k < W; ++k) acc[0] += bget<T>(v, k) * bget<T>(v, k);
    }
    for (long long t = lo + nv * W + threadIdx.x; t < hi; t += blockDim.x) {
      T v = keep ? b * y[t] : (T)0;
#pragma unroll
      for (int l = 0; l < NV; ++l) v += c[l] * src.p[l][t];
      y[t] = v;
      acc[0] += v * v;
    }
  }
  if (want_norm) bred_store<1, T>(bb, acc, 1, false, part, counter, norm + kMaxVecs + 1, kDv);
}

// y_i = f_i x_i with f_i = fac[i * fstride] (inv_sqrt: 1 / sqrt of it); To / Ti casts
template <typename To, typename Ti>
__global__ void bscale_kernel(BatchBlocks bb, To* __restrict__ y, const Ti* __restrict__ x,
                              const double* __restrict__ fac, int fstride, int inv_sqrt,
                              const int* __restrict__ act) {
  const int i = bb.inst[blockIdx.x];
  if (!act[i]) return;
  double f = fac[(size_t)i * fstride];
  if (inv_sqrt) f = f > 0.0 ? 1.0 / sqrt(f) : 0.0;
  const long long lo = bb.lo[blockIdx.x], hi = bb.hi[blockIdx.x];
  if constexpr (sizeof(To) == sizeof(Ti)) {
    const To fs = (To)f;
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) y[e] = fs * (To)x[e];
  } else {
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) y[e] = (To)(f * (double)x[e]);
  }
}

// u_i += f_i x_i (FP64 u, x of type Ti)
template <typename Ti>
__global__ void baxpy64_kernel(BatchBlocks bb, double* __restrict__ u, const Ti* __restrict__ x,
                               const double* __restrict__ fac, const int* __restrict__ act) {
  const int i = bb.inst[blockIdx.x];
  if (!act[i]) return;
  const double f = fac[i];
  const long long lo = bb.lo[blockIdx.x], hi = bb.hi[blockIdx.x];
  for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) u[e] += f * (double)x[e];
}

// per instance: out[i kDv] = |a_i - b_i|^2, out[i kDv + 1] = |a_i|^2
__global__ void __launch_bounds__(kBThreads)
bdiff_kernel(BatchBlocks bb, const double* __restrict__ a, const double* __restrict__ b,
             const int* __restrict__ act, double* part, unsigned* counter, double* out) {
  double acc[2] = {0.0, 0.0};
  const int i = bb.inst[blockIdx.x];
  if (act[i]) {
    for (long long e = bb.lo[blockIdx.x] + threadIdx.x; e < bb.hi[blockIdx.x]; e += blockDim.x) {
      const double d = a[e] - b[e];
      acc[0] += d * d;
      acc[1] += a[e] * a[e];
    }
  }
  bred_store<2, double>(bb, acc, 2, false, part, counter, out, kDv);
}

// Hessenberg column / Givens rotation of step j, one CTA per instance
__global__ void bhcol_kernel(double* hess, HessLayout L, int j, int pass, const double* __restrict__ dv,
                             const int* __restrict__ act) {
  const int i = blockIdx.x;
  if (!act[i]) return;
  hess_column(hess + (size_t)i * L.total(), L, j, pass, dv + (size_t)i * kDv);
}

// ... and marks an instance done when its estimate meets its tolerance
// (or is not finite: the host reports that at the checkpoint)
__global__ void bgivens_kernel(double* hess, HessLayout L, int j, const double* __restrict__ dv,
                               const double* __restrict__ tol, int* act, int* conv, int ninst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst || !act[i]) return;
  const double r = hess_givens(hess + (size_t)i * L.total(), L, j, dv[(size_t)i * kDv + kMaxVecs + 1]);
  if (!(r > tol[i])) {
    act[i] = 0;
    conv[i] = j + 1;
  }
}

// K = K0 (1 + beta sum_a G_a^2) (Picard conductivity, Sec. 2.3)
__global__ void bpicard_k_kernel(const double* __restrict__ K0, const double* __restrict__ G0,
                                 const double* __restrict__ G1, const double* __restrict__ G2, double beta,
                                 double* __restrict__ K, long long n) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    double s = G0[c] * G0[c];
    if (G1) s += G1[c] * G1[c];
    if (G2) s += G2[c] * G2[c];
    K[c] = K0[c] * (1.0 + beta * s);
  }
}

__global__ void brelax_kernel(double* __restrict__ u, const double* __restrict__ u0, double omega, long long n) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    u[c] = omega * u[c] + (1.0 - omega) * u0[c];
}

// ---------------------------------------------------------------------------
// the batched line pass: a persistent grid over the (instance, tile) work list
// ---------------------------------------------------------------------------
struct BPassInst {
  Geom g;
  AxisK<double> a64;
  AxisK<float> a32;
  long long off;      // offset of the instance in the batch vectors
  int tile0, ntiles;  // its work items [tile0, tile0 + ntiles)
};

template <typename T> __device__ __forceinline__ const AxisK<T>& bp_axis(const BPassInst& b);
template <> __device__ __forceinline__ const AxisK<double>& bp_axis<double>(const BPassInst& b) { return b.a64; }
template <> __device__ __forceinline__ const AxisK<float>& bp_axis<float>(const BPassInst& b) { return b.a32; }

// Each CTA takes a contiguous range of work items (so it restages D only
// when its range crosses into the next instance).  kind: apply (first /
// accumulating axis) or derivative.
template <typename T>
__global__ void __launch_bounds__(kBTile * 16)
batch_pass_kernel(const BPassInst* __restrict__ insts, int ninst, int nitems, int axis, int kind,
                  const T* __restrict__ K, const T* __restrict__ u, T* __restrict__ out,
                  const int* __restrict__ act) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w0 = (int)((long long)nitems * blockIdx.x / gridDim.x);
  const int w1 = (int)((long long)nitems * (blockIdx.x + 1) / gridDim.x);
  if (w0 >= w1) return;
  // instance of item w0: the last one with tile0 <= w0
  int ii = 0, hi = ninst - 1;
  while (ii < hi) {
    const int mid = (ii + hi + 1) >> 1;
    if (insts[mid].tile0 <= w0) ii = mid;
    else hi = mid - 1;
  }
  int cur = -1;
  PassSmem<T> sm;
  for (int w = w0; w < w1; ++w) {
    while (ii + 1 < ninst && insts[ii + 1].tile0 <= w) ++ii;
    const BPassInst& b = insts[ii];
    if (w - b.tile0 >= b.ntiles || !act[ii]) continue;  // uniform over the CTA
    const AxisK<T>& ax = bp_axis<T>(b);
    if (ii != cur) {
      __syncthreads();  // the previous instance's tables are no longer read
      sm = pass_stage<T, CHEB_ROUTE_DENSE, 0, kBTile>(smem_raw, ax);
      cur = ii;
    }
    line_pass_tile<T, CHEB_ROUTE_DENSE, 0, 1, kBTile>(b.g, axis, kind, ax, K ? K + b.off : nullptr, u + b.off,
                                                     out + b.off, nullptr, w - b.tile0, sm);
    __syncthreads();  // the tile buffers are reused by the next item
  }
}

// ---------------------------------------------------------------------------
// the engine
// ---------------------------------------------------------------------------
template <typename T>
struct BBufs {
  int nvec = 0, kaug = 0;
  T* V = nullptr;    // nvec x total
  T* Z = nullptr;    // kaug x total
  T* BZ = nullptr;   // kaug x total
  T* tmp = nullptr;
  T* x = nullptr;
  T* c = nullptr;
  T* K = nullptr;
};

struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  long long nkernels = 0;
};

struct Engine {
  int B = 0;
  std::vector<cheb_plan_s*> plans;
  std::vector<Fdm*> fdm;
  std::vector<long long> off, len;
  long long total = 0;
  int nmax = 0;          // largest axis size
  cudaStream_t s = nullptr;
  std::vector<cudaStream_t> bs;  // one branch stream per instance
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  // vector-kernel block tables
  BatchBlocks bb{};
  int* d_inst = nullptr;
  long long* d_lo = nullptr;
  long long* d_hi = nullptr;
  int* d_first = nullptr;
  double* part = nullptr;
  unsigned* counter = nullptr;
  // line-pass work lists per axis
  BPassInst* d_pass[3] = {nullptr, nullptr, nullptr};
  int nitems[3] = {0, 0, 0};
  int pass_grid[2][3] = {{0, 0, 0}, {0, 0, 0}};
  size_t pass_smem[2] = {0, 0};
  int dim = 3;
  // per-instance device state
  double* dv = nullptr;      // B x kDv
  double* hv = nullptr;      // pinned mirror
  int* act = nullptr;        // stepping mask (cleared by bgivens)
  int* cyc = nullptr;        // cycle / solve mask
  int* conv = nullptr;       // step at which bgivens cleared the mask
  int* hact = nullptr;       // pinned read-back mirrors
  int* hconv = nullptr;
  double* tol = nullptr;     // per-instance tolerance
  double* coef = nullptr;    // per-instance coefficient rows (device)
  double* fac = nullptr;     // per-instance factors (device)
  double* hess = nullptr;    // B Hessenberg blocks
  double* hhess = nullptr;
  int hess_nb = 0;
  BBufs<float> b32;
  BBufs<double> b64;
  double* r64 = nullptr;
  std::vector<double> kref;
  int precond = CHEB_PRECOND_FDM;
  FdmBatch* fb = nullptr;           // batched lift / face / boundary-line steps (FP32)
  std::vector<char> in_fb;          // instance i runs its FP32 preconditioner through fb
  std::map<std::string, StepGraph> graphs;
  bool warm = false;
  int captures = 0;

  ~Engine() { release(); }
  void release() {
    for (auto& kv : graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
    fdm_batch_free(fb);
    fb = nullptr;
    auto fr = [](auto*& p) { if (p) cudaFree(p); p = nullptr; };
    auto frh = [](auto*& p) { if (p) cudaFreeHost(p); p = nullptr; };
    fr(d_inst); fr(d_lo); fr(d_hi); fr(d_first); fr(part); fr(counter);
    for (auto& d : d_pass) fr(d);
    fr(dv); fr(act); fr(cyc); fr(conv); fr(tol); fr(coef); fr(fac); fr(hess); fr(r64);
    frh(hv); frh(hact); frh(hconv); frh(hhess);
    fr(b32.V); fr(b32.Z); fr(b32.BZ); fr(b32.tmp); fr(b32.x); fr(b32.c); fr(b32.K);
    fr(b64.V); fr(b64.Z); fr(b64.BZ); fr(b64.tmp); fr(b64.x); fr(b64.c); fr(b64.K);
    for (auto& st : bs) if (st) cudaStreamDestroy(st);
    bs.clear();
    for (auto& e : join) if (e) cudaEventDestroy(e);
    join.clear();
    if (fork) cudaEventDestroy(fork);
    fork = nullptr;
    if (s) cudaStreamDestroy(s);
    s = nullptr;
  }
};

template <typename T> BBufs<T>& bufs_of(Engine& E);
template <> BBufs<float>& bufs_of<float>(Engine& E) { return E.b32; }
template <> BBufs<double>& bufs_of<double>(Engine& E) { return E.b64; }

int grid1(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 148 * 8)); }

int engine_setup(Engine& E, int count, const cheb_plan* plans, int precond) {
  E.B = count;
  E.precond = precond;
  E.plans.assign(plans, plans + count);
  E.dim = E.plans[0]->dim;
  for (auto* p : E.plans) {
    if (p->dim != E.dim) { set_error("batched plans must have the same dimension"); return CHEB_ERR_ARG; }
    for (int a = 0; a < p->dim; ++a)
      if (!p->ax[a].dense_ok) { set_error("lockstep batches need n <= 129 on every axis"); return CHEB_ERR_UNSUPPORTED; }
  }
  CHEB_CUDA(cudaStreamCreateWithFlags(&E.s, cudaStreamNonBlocking));
  CHEB_CUDA(cudaEventCreateWithFlags(&E.fork, cudaEventDisableTiming));
  E.bs.assign(count, nullptr);
  E.join.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    CHEB_CUDA(cudaStreamCreateWithFlags(&E.bs[i], cudaStreamNonBlocking));
    CHEB_CUDA(cudaEventCreateWithFlags(&E.join[i], cudaEventDisableTiming));
  }
  // layout
  E.off.resize(count);
  E.len.resize(count);
  long long o = 0;
  for (int i = 0; i < count; ++i) {
    E.off[i] = o;
    E.len[i] = (long long)E.plans[i]->size();
    o += (E.len[i] + kBAlign - 1) / kBAlign * kBAlign;
    for (int a = 0; a < E.dim; ++a) E.nmax = std::max(E.nmax, E.plans[i]->n[a]);
  }
  E.total = std::max<long long>(o, kBAlign);
  // vector-kernel blocks
  std::vector<int> inst, first(count + 1, 0);
  std::vector<long long> lo, hi;
  for (int i = 0; i < count; ++i) {
    first[i] = (int)inst.size();
    for (long long c = 0; c < E.len[i]; c += kBChunk) {
      inst.push_back(i);
      lo.push_back(E.off[i] + c);
      hi.push_back(E.off[i] + std::min(E.len[i], c + kBChunk));
    }
  }
  first[count] = (int)inst.size();
  const int nblk = (int)inst.size();
  CHEB_CUDA(cudaMalloc(&E.d_inst, sizeof(int) * nblk));
  CHEB_CUDA(cudaMalloc(&E.d_lo, sizeof(long long) * nblk));
  CHEB_CUDA(cudaMalloc(&E.d_hi, sizeof(long long) * nblk));
  CHEB_CUDA(cudaMalloc(&E.d_first, sizeof(int) * (count + 1)));
  CHEB_CUDA(cudaMemcpy(E.d_inst, inst.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice));
  CHEB_CUDA(cudaMemcpy(E.d_lo, lo.data(), sizeof(long long) * nblk, cudaMemcpyHostToDevice));
  CHEB_CUDA(cudaMemcpy(E.d_hi, hi.data(), sizeof(long long) * nblk, cudaMemcpyHostToDevice));
  CHEB_CUDA(cudaMemcpy(E.d_first, first.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice));
  E.bb = BatchBlocks{E.d_inst, E.d_lo, E.d_hi, E.d_first, nblk, count};
  CHEB_CUDA(cudaMalloc(&E.part, sizeof(double) * (kMaxVecs + 1) * (size_t)nblk));
  CHEB_CUDA(cudaMalloc(&E.counter, sizeof(unsigned)));
  CHEB_CUDA(cudaMemset(E.counter, 0, sizeof(unsigned)));
  // line-pass work lists
  for (int a = 0; a < E.dim; ++a) {
    std::vector<BPassInst> v(count);
    int items = 0;
    for (int i = 0; i < count; ++i) {
      const cheb_plan_s* p = E.plans[i];
      BPassInst& b = v[i];
      std::memset(&b, 0, sizeof(b));
      b.g = p->geom();
      const AxisTables& t = p->ax[a];
      b.a64.n = t.n; b.a64.N = t.N; b.a64.scale = t.scale; b.a64.D = t.D64;
      b.a32.n = t.n; b.a32.N = t.N; b.a32.scale = (float)t.scale; b.a32.D = t.D32;
      b.off = E.off[i];
      b.tile0 = items;
      b.ntiles = a == 0 ? (p->n[1] * p->n[2] + kBTile - 1) / kBTile
                        : ((p->n[0] + kBTile - 1) / kBTile) * (a == 1 ? p->n[2] : p->n[1]);
      items += b.ntiles;
    }
    E.nitems[a] = items;
    CHEB_CUDA(cudaMalloc(&E.d_pass[a], sizeof(BPassInst) * count));
    CHEB_CUDA(cudaMemcpy(E.d_pass[a], v.data(), sizeof(BPassInst) * count, cudaMemcpyHostToDevice));
  }
  // per-instance state
  CHEB_CUDA(cudaMalloc(&E.dv, sizeof(double) * kDv * count));
  CHEB_CUDA(cudaMallocHost(&E.hv, sizeof(double) * kDv * count));
  CHEB_CUDA(cudaMalloc(&E.act, sizeof(int) * count));
  CHEB_CUDA(cudaMalloc(&E.cyc, sizeof(int) * count));
  CHEB_CUDA(cudaMalloc(&E.conv, sizeof(int) * count));
  CHEB_CUDA(cudaMallocHost(&E.hact, sizeof(int) * count));
  CHEB_CUDA(cudaMallocHost(&E.hconv, sizeof(int) * count));
  CHEB_CUDA(cudaMalloc(&E.tol, sizeof(double) * count));
  CHEB_CUDA(cudaMalloc(&E.coef, sizeof(double) * kMaxVecs * count));
  CHEB_CUDA(cudaMalloc(&E.fac, sizeof(double) * count));
  // preconditioner tables of every plan
  E.fdm.assign(count, nullptr);
  if (precond == CHEB_PRECOND_FDM)
    for (int i = 0; i < count; ++i) {
      int st;
      if ((st = plan_fdm(E.plans[i], &E.fdm[i]))) return st;
      if ((st = fdm_clear(*E.fdm[i], E.s))) return st;
    }
  E.kref.assign(count, 1.0);
  return CHEB_OK;
}

template <typename T>
int ensure_bbufs(Engine& E, int nvec, int kaug) {
  BBufs<T>& b = bufs_of<T>(E);
  if (b.nvec >= nvec && b.kaug >= kaug) return CHEB_OK;
  auto fr = [](T*& p) { if (p) cudaFree(p); p = nullptr; };
  fr(b.V); fr(b.Z); fr(b.BZ);
  const size_t tb = sizeof(T) * (size_t)E.total;
  CHEB_CUDA(cudaMalloc(&b.V, tb * nvec));
  CHEB_CUDA(cudaMalloc(&b.Z, tb * std::max(1, kaug)));
  CHEB_CUDA(cudaMalloc(&b.BZ, tb * std::max(1, kaug)));
  // zero: the gaps between instances are read by no kernel, but stay finite
  CHEB_CUDA(cudaMemsetAsync(b.V, 0, tb * nvec, E.s));
  CHEB_CUDA(cudaMemsetAsync(b.Z, 0, tb * std::max(1, kaug), E.s));
  CHEB_CUDA(cudaMemsetAsync(b.BZ, 0, tb * std::max(1, kaug), E.s));
  if (!b.tmp) {
    CHEB_CUDA(cudaMalloc(&b.tmp, tb));
    CHEB_CUDA(cudaMalloc(&b.x, tb));
    CHEB_CUDA(cudaMalloc(&b.c, tb));
    CHEB_CUDA(cudaMalloc(&b.K, tb));
    CHEB_CUDA(cudaMemsetAsync(b.tmp, 0, tb, E.s));
    CHEB_CUDA(cudaMemsetAsync(b.x, 0, tb, E.s));
    CHEB_CUDA(cudaMemsetAsync(b.c, 0, tb, E.s));
    CHEB_CUDA(cudaMemsetAsync(b.K, 0, tb, E.s));
  }
  b.nvec = nvec;
  b.kaug = kaug;
  return CHEB_OK;
}

// ---- launch helpers ----
template <typename T>
int bpass(Engine& E, int axis, int kind, const T* K, const T* u, T* out, cudaStream_t s) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  auto kern = batch_pass_kernel<T>;
  if (!E.pass_grid[pi][axis]) {
    const size_t smem = pass_smem_bytes<T>(CHEB_ROUTE_DENSE, E.nmax, 0, kBTile);
    int st;
    if ((st = ensure_smem_attr((const void*)kern, smem))) return st;
    int occ = 0;
    CHEB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBTile * 16, smem));
    int dev = 0, sms = 0;
    CHEB_CUDA(cudaGetDevice(&dev));
    CHEB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    E.pass_smem[pi] = smem;
    E.pass_grid[pi][axis] = std::max(1, std::min(E.nitems[axis], sms * std::max(1, occ)));
  }
  kern<<<E.pass_grid[pi][axis], kBTile * 16, E.pass_smem[pi], s>>>(E.d_pass[axis], E.B, E.nitems[axis], axis, kind,
                                                                    K, u, out, E.act);
  CHEB_LAUNCH_CHECK("batch_pass_kernel");
  return CHEB_OK;
}

template <typename T>
int bapply(Engine& E, const T* K, const T* u, T* out, cudaStream_t s) {
  int st;
  for (int a = 0; a < E.dim; ++a)
    if ((st = bpass<T>(E, a, a == 0 ? kApplyFirst : kApplyAcc, K, u, out, s))) return st;
  return CHEB_OK;
}

// z = M^{-1} r for the live instances, one graph branch (stream) each
// z = M^{-1} r for the live instances.  FP32 with the batched steps: one
// lift launch for all instances, then each instance's two tcgen05 sweeps
// as a branch, then one face launch and the boundary-line launches for all
// instances; other instances run their whole preconditioner in their branch.
template <typename T>
int bprecond(Engine& E, const std::vector<int>& live, const T* r, T* z, cudaStream_t s) {
  if (E.precond != CHEB_PRECOND_FDM) {
    CHEB_CUDA(cudaMemcpyAsync(z, r, sizeof(T) * (size_t)E.total, cudaMemcpyDeviceToDevice, s));
    return CHEB_OK;
  }
  int st = CHEB_OK;
  bool batched = false;
  if constexpr (sizeof(T) == 4) {
    batched = E.fb != nullptr;
    if (batched && (st = fdm_batch_lift(E.fb, r, s))) return st;
  }
  CHEB_CUDA(cudaEventRecord(E.fork, s));
  for (int i : live) {
    CHEB_CUDA(cudaStreamWaitEvent(E.bs[i], E.fork, 0));
    if constexpr (sizeof(T) == 4) {
      if (batched && E.in_fb[i]) st = fdm_rot_core(E.plans[i], *E.fdm[i], E.kref[i], r + E.off[i], z + E.off[i], E.bs[i]);
      else st = fdm_apply<T>(E.plans[i], *E.fdm[i], E.kref[i], r + E.off[i], z + E.off[i], E.bs[i]);
    } else {
      st = fdm_apply<T>(E.plans[i], *E.fdm[i], E.kref[i], r + E.off[i], z + E.off[i], E.bs[i]);
    }
    if (st) return st;
    CHEB_CUDA(cudaEventRecord(E.join[i], E.bs[i]));
  }
  for (int i : live) CHEB_CUDA(cudaStreamWaitEvent(s, E.join[i], 0));
  if constexpr (sizeof(T) == 4) {
    if (batched && (st = fdm_batch_faces(E.fb, r, z, s))) return st;
  }
  return CHEB_OK;
}

template <typename T>
int bop_B(Engine& E, const std::vector<int>& live, const T* K, const T* v, T* out, T* tmp, cudaStream_t s) {
  int st;
  if ((st = bapply<T>(E, K, v, tmp, s))) return st;
  return bprecond<T>(E, live, tmp, out, s);
}

template <typename T>
int bmdot(Engine& E, const T* const* src, int cnt, const T* w, bool with_self, const int* mask, cudaStream_t s) {
  VecList<T> vl;
  for (int l = 0; l < kMaxVecs; ++l) vl.p[l] = l < cnt ? src[l] : nullptr;
  return count_dispatch(cnt, [&](auto c) -> int {
    bmdot_kernel<T, decltype(c)::value><<<E.bb.nblk, kBThreads, 0, s>>>(E.bb, vl, w, with_self ? 1 : 0, mask,
                                                                        E.part, E.counter, E.dv);
    CHEB_LAUNCH_CHECK("bmdot_kernel");
    return CHEB_OK;
  });
}

// y = beta y + sum_l c_l src_l: coefficients from dv (dev, sign) or from the
// host matrix hmat[i * cnt + l] (copied to the device first)
template <typename T>
int bmaxpy(Engine& E, const T* const* src, int cnt, bool from_dv, double sign, const double* hmat, double beta,
           T* y, const int* mask, bool want_norm, cudaStream_t s) {
  if (cnt < 0 || cnt > kMaxVecs) { set_error("bad vector count in a batched multi-axpy"); return CHEB_ERR_ARG; }
  VecList<T> vl;
  for (int l = 0; l < kMaxVecs; ++l) vl.p[l] = l < cnt ? src[l] : nullptr;
  const double* cm = nullptr;
  if (!from_dv) {
    // pageable source: the copy is staged before the call returns, so the
    // caller's matrix may change right after (never called under capture)
    CHEB_CUDA(cudaMemcpyAsync(E.coef, hmat, sizeof(double) * (size_t)E.B * cnt, cudaMemcpyHostToDevice, s));
    cm = E.coef;
  }
  return count_dispatch(cnt, [&](auto c) -> int {
    bmaxpy_kernel<T, decltype(c)::value><<<E.bb.nblk, kBThreads, 0, s>>>(
        E.bb, vl, from_dv ? E.dv : nullptr, sign, cm, beta, y, mask, want_norm ? 1 : 0, E.part, E.counter, E.dv);
    CHEB_LAUNCH_CHECK("bmaxpy_kernel");
    return CHEB_OK;
  });
}

// y = f_i x with host factors f (copied to the device)
template <typename To, typename Ti>
int bscale_host(Engine& E, To* y, const Ti* x, const std::vector<double>& f, const int* mask, cudaStream_t s) {
  CHEB_CUDA(cudaMemcpyAsync(E.fac, f.data(), sizeof(double) * E.B, cudaMemcpyHostToDevice, s));
  bscale_kernel<To, Ti><<<E.bb.nblk, 256, 0, s>>>(E.bb, y, x, E.fac, 1, 0, mask);
  CHEB_LAUNCH_CHECK("bscale_kernel");
  return CHEB_OK;
}

int sync_hv(Engine& E, int rows) {
  CHEB_CUDA(cudaMemcpyAsync(E.hv, E.dv, sizeof(double) * kDv * E.B, cudaMemcpyDeviceToHost, E.s));
  (void)rows;
  CHEB_CUDA(cudaStreamSynchronize(E.s));
  return CHEB_OK;
}

// small uploads come from pageable vectors: staged before the call returns
int upload_mask(Engine& E, int* dmask, const std::vector<int>& live, cudaStream_t s) {
  std::vector<int> m(E.B, 0);
  for (int i : live) m[i] = 1;
  CHEB_CUDA(cudaMemcpyAsync(dmask, m.data(), sizeof(int) * E.B, cudaMemcpyHostToDevice, s));
  return CHEB_OK;
}

// ---------------------------------------------------------------------------
// lockstep LGMRES(m, k) on B z = c for the live instances (x: initial guess
// unless x_zero; tol: per-instance absolute tolerances on |c - B x|)
// ---------------------------------------------------------------------------
struct BStats {
  std::vector<int> iterations, cycles, applies, status;
  std::vector<double> resid;
  int syncs = 0;
  void init(int B) {
    iterations.assign(B, 0);
    cycles.assign(B, 0);
    applies.assign(B, 0);
    status.assign(B, CHEB_ERR_NOT_CONVERGED);
    resid.assign(B, 0.0);
  }
};

template <typename T>
int blgmres(Engine& E, std::vector<int> live, int m, int k, int maxiter, const std::vector<double>& tol,
            const T* K, const T* c, T* x, bool x_zero, BStats& stt) {
  cudaStream_t s = E.s;
  const int nb = m + k + 1;
  int st;
  if ((st = ensure_bbufs<T>(E, nb, std::max(1, k)))) return st;
  BBufs<T>& Bf = bufs_of<T>(E);
  const size_t ld = (size_t)E.total;
  auto Vp = [&](int i) { return Bf.V + (size_t)i * ld; };
  auto Zp = [&](int i) { return Bf.Z + (size_t)i * ld; };
  auto BZp = [&](int i) { return Bf.BZ + (size_t)i * ld; };
  const HessLayout L{nb};
  if (E.hess_nb < nb) {
    if (E.hess) cudaFree(E.hess);
    if (E.hhess) cudaFreeHost(E.hhess);
    CHEB_CUDA(cudaMalloc(&E.hess, sizeof(double) * L.total() * E.B));
    CHEB_CUDA(cudaMallocHost(&E.hhess, sizeof(double) * L.total() * E.B));
    E.hess_nb = nb;
  }
  CHEB_CUDA(cudaMemcpyAsync(E.tol, tol.data(), sizeof(double) * E.B, cudaMemcpyHostToDevice, s));
  int naug = 0, next_slot = 0;
  bool zero = x_zero;
  std::vector<double> y(nb), g(nb + 1);
  while (!live.empty()) {
    // ---- r = c - B x into V0, norms
    if ((st = upload_mask(E, E.act, live, s))) return st;
    if (zero) {
      CHEB_CUDA(cudaMemcpyAsync(Vp(0), c, sizeof(T) * ld, cudaMemcpyDeviceToDevice, s));
    } else {
      if ((st = bop_B<T>(E, live, K, x, Vp(0), Bf.tmp, s))) return st;
      for (int i : live) stt.applies[i]++;
      if ((st = k_residual<T>(Vp(0), c, ld, s))) return st;
    }
    const T* v0 = Vp(0);
    if ((st = bmdot<T>(E, &v0, 0, Vp(0), true, E.act, s))) return st;
    if ((st = sync_hv(E, 1))) return st;
    stt.syncs++;
    std::vector<int> next;
    std::vector<double> beta(E.B, 0.0), inv(E.B, 0.0);
    for (int i : live) {
      const double bt = std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv + 0]));
      stt.resid[i] = bt;
      if (!std::isfinite(bt)) { set_error("non-finite residual in a batched solve"); return CHEB_ERR_NONFINITE; }
      if (bt <= tol[i]) { stt.status[i] = CHEB_OK; continue; }
      if (stt.iterations[i] >= maxiter) { stt.status[i] = CHEB_ERR_NOT_CONVERGED; continue; }
      beta[i] = bt;
      inv[i] = 1.0 / bt;
      next.push_back(i);
    }
    live = next;
    if (live.empty()) break;
    if ((st = upload_mask(E, E.act, live, s))) return st;
    if ((st = upload_mask(E, E.cyc, live, s))) return st;
    if ((st = bscale_host<T, T>(E, Vp(0), Vp(0), inv, E.act, s))) return st;
    for (int i : live) stt.cycles[i]++;
    // ---- Hessenberg blocks: g[0] = beta_i
    {
      std::vector<double> h0(L.total() * E.B, 0.0);
      for (int i : live) h0[(size_t)i * L.total() + L.g()] = beta[i];
      CHEB_CUDA(cudaMemcpyAsync(E.hess, h0.data(), sizeof(double) * h0.size(), cudaMemcpyHostToDevice, s));
      CHEB_CUDA(cudaMemsetAsync(E.conv, 0, sizeof(int) * E.B, s));
    }
    const int m_eff = m + (k - naug);
    int budget = m_eff + naug;
    for (int i : live) budget = std::min(budget, std::max(1, maxiter - stt.iterations[i]));
    // captured steps launch every instance's preconditioner branch; the
    // device mask (E.act) skips the finished ones, so one graph per
    // (precision, step, augmentation slot) serves every live set
    std::vector<int> all(E.B);
    for (int i = 0; i < E.B; ++i) all[i] = i;
    // ---- Arnoldi steps, one graph replay each
    int steps_run = 0;
    for (int j = 0; j < budget; ++j) {
      const int slot = j < m_eff ? -1 : (next_slot - naug + (j - m_eff) + 4 * k) % k;
      auto step = [&](cudaStream_t cs, const std::vector<int>& branches) -> int {
        int r;
        T* wv = Vp(j + 1);
        if (j < m_eff) {
          if ((r = bop_B<T>(E, branches, K, Vp(j), wv, Bf.tmp, cs))) return r;
        } else {
          CHEB_CUDA(cudaMemcpyAsync(wv, BZp(slot), sizeof(T) * ld, cudaMemcpyDeviceToDevice, cs));
        }
        const T* src[kMaxVecs];
        for (int i = 0; i <= j; ++i) src[i] = Vp(i);
        if ((r = bmdot<T>(E, src, j + 1, wv, false, E.act, cs))) return r;
        if ((r = bmaxpy<T>(E, src, j + 1, true, -1.0, nullptr, 1.0, wv, E.act, true, cs))) return r;
        bhcol_kernel<<<E.B, 64, 0, cs>>>(E.hess, L, j, 0, E.dv, E.act);
        CHEB_LAUNCH_CHECK("bhcol_kernel");
        bscale_kernel<T, T><<<E.bb.nblk, 256, 0, cs>>>(E.bb, wv, wv, E.dv + kMaxVecs + 1, kDv, 1, E.act);
        CHEB_LAUNCH_CHECK("bscale_kernel");
        bgivens_kernel<<<(E.B + 31) / 32, 32, 0, cs>>>(E.hess, L, j, E.dv, E.tol, E.act, E.conv, E.B);
        CHEB_LAUNCH_CHECK("bgivens_kernel");
        return CHEB_OK;
      };
      if (!E.warm) {
        // first step of the engine runs eagerly (lazy allocations, kernel attributes)
        if ((st = step(s, live))) return st;
        CHEB_CUDA(cudaStreamSynchronize(s));
        E.warm = true;
      } else {
        const std::string key = std::to_string(sizeof(T)) + "|" + std::to_string(j) + "|" + std::to_string(slot) +
                                "|" + std::to_string(m_eff);
        StepGraph& gr = E.graphs[key];
        if (!gr.exec) {
          const long long l0 = thread_launches();
          CHEB_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
          const int r = step(s, all);
          cudaGraph_t graph = nullptr;
          const cudaError_t ce = cudaStreamEndCapture(s, &graph);
          if (r) { if (graph) cudaGraphDestroy(graph); return r; }
          if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
          const cudaError_t ie = cudaGraphInstantiate(&gr.exec, graph, 0);
          cudaGraphDestroy(graph);
          if (ie != cudaSuccess) { gr.exec = nullptr; return cuda_fail(ie, "cudaGraphInstantiate"); }
          gr.nkernels = thread_launches() - l0;
          add_launches(-gr.nkernels);  // recorded, not run: counted at each replay
          E.captures++;
        }
        CHEB_CUDA(cudaGraphLaunch(gr.exec, s));
        add_launches(gr.nkernels);
      }
      for (int i : live) stt.applies[i] += j < m_eff ? 1 : 0;
      steps_run = j + 1;
      // every 8 steps: stop the cycle early once every instance has converged
      if ((j + 1) % 8 == 0 && j + 1 < budget) {
        CHEB_CUDA(cudaMemcpyAsync(E.hact, E.act, sizeof(int) * E.B, cudaMemcpyDeviceToHost, s));
        CHEB_CUDA(cudaStreamSynchronize(s));
        stt.syncs++;
        bool any = false;
        for (int i : live) any |= E.hact[i] != 0;
        if (!any) break;
      }
    }
    // ---- checkpoint: every instance's Hessenberg block and convergence step
    CHEB_CUDA(cudaMemcpyAsync(E.hhess, E.hess, sizeof(double) * L.total() * E.B, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaMemcpyAsync(E.hconv, E.conv, sizeof(int) * E.B, cudaMemcpyDeviceToHost, s));
    CHEB_CUDA(cudaStreamSynchronize(s));
    stt.syncs++;
    std::vector<double> cmat((size_t)E.B * nb, 0.0), hy((size_t)E.B * (nb + 1), 0.0);
    int cnt_max = 0;
    std::vector<int> steps_of(E.B, 0);
    for (int i : live) {
      const double* hh = E.hhess + (size_t)i * L.total();
      const int steps = E.hconv[i] > 0 ? E.hconv[i] : steps_run;
      for (int q = 0; q < steps; ++q)
        if (!std::isfinite(hh[L.res() + q])) {
          set_error("non-finite Arnoldi residual in a batched solve");
          return CHEB_ERR_NONFINITE;
        }
      steps_of[i] = steps;
      stt.iterations[i] += steps;
      cnt_max = std::max(cnt_max, steps);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta[i];
      for (int q = 0; q < steps; ++q) {
        const double cq = hh[L.cs() + q], sq = hh[L.sn() + q];
        g[q + 1] = -sq * g[q];
        g[q] = cq * g[q];
      }
      for (int q = steps - 1; q >= 0; --q) {
        double t = g[q];
        for (int l = q + 1; l < steps; ++l) t -= hh[L.R() + (size_t)q * nb + l] * y[l];
        const double d = hh[L.R() + (size_t)q * nb + q];
        y[q] = d != 0.0 ? t / d : 0.0;
      }
      for (int q = 0; q < steps; ++q) cmat[(size_t)i * nb + q] = y[q];
      for (int q = 0; q <= steps; ++q) {
        double t = 0.0;
        for (int l = 0; l < steps; ++l)
          if (q <= l + 1) t += hh[L.H() + (size_t)q * nb + l] * y[l];
        hy[(size_t)i * (nb + 1) + q] = t;
      }
    }
    // ---- dx = W y per instance (coefficient rows of cnt_max), x += dx
    if ((st = upload_mask(E, E.cyc, live, s))) return st;
    {
      const T* src[kMaxVecs];
      for (int q = 0; q < cnt_max; ++q)
        src[q] = q < m_eff ? Vp(q) : Zp((next_slot - naug + (q - m_eff) + 4 * k) % k);
      std::vector<double> cm((size_t)E.B * cnt_max, 0.0);
      for (int i : live)
        for (int q = 0; q < steps_of[i]; ++q) cm[(size_t)i * cnt_max + q] = cmat[(size_t)i * nb + q];
      if ((st = bmaxpy<T>(E, src, cnt_max, false, 1.0, cm.data(), 0.0, Bf.tmp, E.cyc, k > 0, s))) return st;
      if (zero) {
        std::vector<double> one(E.B, 1.0);
        if ((st = bscale_host<T, T>(E, x, Bf.tmp, one, E.cyc, s))) return st;
      } else {
        const T* t1[1] = {Bf.tmp};
        std::vector<double> ones(E.B, 1.0);
        if ((st = bmaxpy<T>(E, t1, 1, false, 1.0, ones.data(), 1.0, x, E.cyc, false, s))) return st;
      }
      zero = false;
    }
    // ---- augmentation: z = dx / |dx|, B z = V Hbar y / |dx| (linearity)
    if (k > 0) {
      if ((st = sync_hv(E, kMaxVecs + 2))) return st;
      stt.syncs++;
      std::vector<double> invdx(E.B, 0.0);
      std::vector<double> hm((size_t)E.B * (cnt_max + 1), 0.0);
      for (int i : live) {
        const double dxn = std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv + kMaxVecs + 1]));
        invdx[i] = dxn > 0 ? 1.0 / dxn : 0.0;
        for (int q = 0; q <= steps_of[i]; ++q)
          hm[(size_t)i * (cnt_max + 1) + q] = hy[(size_t)i * (nb + 1) + q] * invdx[i];
      }
      if ((st = bscale_host<T, T>(E, Zp(next_slot), Bf.tmp, invdx, E.cyc, s))) return st;
      const T* vs[kMaxVecs];
      for (int q = 0; q <= cnt_max; ++q) vs[q] = Vp(q);
      if ((st = bmaxpy<T>(E, vs, cnt_max + 1, false, 1.0, hm.data(), 0.0, BZp(next_slot), E.cyc, false, s)))
        return st;
      next_slot = (next_slot + 1) % k;
      naug = std::min(naug + 1, k);
    }
  }
  CHEB_CUDA(cudaStreamSynchronize(s));
  return CHEB_OK;
}

// ---------------------------------------------------------------------------
// lockstep solves of A_i u_i = b_i (FP64, or FP32 inner LGMRES inside FP64
// refinement), for the instances in `live`
// ---------------------------------------------------------------------------
int bsolve(Engine& E, std::vector<int> live, const cheb_solve_opts& o, const double* K, const double* b, double* u,
           std::vector<cheb_solve_info>& info, bool kref_fixed) {
  cudaStream_t s = E.s;
  int st;
  if (!kref_fixed)
    for (int i : live) {
      if (o.kref > 0) E.kref[i] = o.kref;
      else if ((st = plan_kref(E.plans[i], K + E.off[i], &E.kref[i], s))) return st;
    }
  for (int i : live) info[i].kref = E.kref[i];
  // every instance's preconditioner is a branch of the captured steps: make
  // its first-use allocations before any capture
  if (E.precond == CHEB_PRECOND_FDM)
    for (int i = 0; i < E.B; ++i) {
      st = o.mode == CHEB_SOLVE_FP64 ? fdm_prepare<double>(E.plans[i], *E.fdm[i], s)
                                     : fdm_prepare<float>(E.plans[i], *E.fdm[i], s);
      if (st) return st;
    }
  // FP32: the lift, face and boundary-line steps of the instances with the
  // tcgen05 route run batched (their per-instance kref in the work list)
  if (E.precond == CHEB_PRECOND_FDM && o.mode == CHEB_SOLVE_MIXED) {
    if (!E.fb) {
      std::vector<const cheb_plan_s*> bp;
      std::vector<Fdm*> bf;
      std::vector<long long> bo;
      E.in_fb.assign(E.B, 0);
      for (int i = 0; i < E.B; ++i)
        if (fdm_batchable(E.plans[i], *E.fdm[i])) {
          E.in_fb[i] = 1;
          bp.push_back(E.plans[i]);
          bf.push_back(E.fdm[i]);
          bo.push_back(E.off[i]);
        }
      if (!bp.empty() && (st = fdm_batch_create(&E.fb, bp, bf, bo))) return st;
    }
    if (E.fb) {
      std::vector<double> kb;
      for (int i = 0; i < E.B; ++i)
        if (E.in_fb[i]) kb.push_back(E.kref[i]);
      if ((st = fdm_batch_kref(E.fb, kb))) return st;
    }
  }
  const long long n = E.total;
  BStats stt;
  stt.init(E.B);
  if (o.mode == CHEB_SOLVE_FP64) {
    if ((st = ensure_bbufs<double>(E, o.restart + o.augment + 1, std::max(1, o.augment)))) return st;
    BBufs<double>& Bf = E.b64;
    if ((st = upload_mask(E, E.act, live, s))) return st;
    if ((st = bprecond<double>(E, live, b, Bf.c, s))) return st;
    const double* cc = Bf.c;
    if ((st = bmdot<double>(E, &cc, 0, Bf.c, true, E.act, s))) return st;
    if ((st = sync_hv(E, 1))) return st;
    std::vector<double> nb(E.B, 0.0), tol(E.B, 0.0);
    std::vector<int> go;
    for (int i : live) {
      nb[i] = std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv]));
      if (nb[i] == 0.0) {
        CHEB_CUDA(cudaMemsetAsync(u + E.off[i], 0, sizeof(double) * E.len[i], s));
        info[i].status = CHEB_OK;
        continue;
      }
      tol[i] = std::max(o.rtol * nb[i], o.atol);
      go.push_back(i);
    }
    if ((st = blgmres<double>(E, go, o.restart, o.augment, o.maxiter, tol, K, Bf.c, u, false, stt))) return st;
    for (int i : go) {
      info[i].iterations += stt.iterations[i];
      info[i].cycles += stt.cycles[i];
      info[i].applies_fp64 += stt.applies[i];
      info[i].rel_residual = stt.resid[i] / nb[i];
      info[i].status = stt.status[i];
    }
    return CHEB_OK;
  }
  // ---- mixed
  if ((st = ensure_bbufs<float>(E, o.restart + o.augment + 1, std::max(1, o.augment)))) return st;
  BBufs<float>& Bf = E.b32;
  if (!E.r64) CHEB_CUDA(cudaMalloc(&E.r64, sizeof(double) * (size_t)n));
  if ((st = k_cast_scale<float, double>(Bf.K, K, 1.0, (size_t)n, s))) return st;
  if ((st = upload_mask(E, E.act, live, s))) return st;
  std::vector<double> nb(E.B, 0.0);
  {
    if ((st = bmdot<double>(E, &b, 0, b, true, E.act, s))) return st;
    if ((st = sync_hv(E, 1))) return st;
    std::vector<double> sb(E.B, 0.0), isb(E.B, 0.0);
    std::vector<int> go;
    for (int i : live) {
      sb[i] = std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv]));
      if (sb[i] == 0.0) {
        CHEB_CUDA(cudaMemsetAsync(u + E.off[i], 0, sizeof(double) * E.len[i], s));
        info[i].status = CHEB_OK;
        continue;
      }
      isb[i] = 1.0 / sb[i];
      go.push_back(i);
    }
    live = go;
    if (live.empty()) return CHEB_OK;
    if ((st = upload_mask(E, E.act, live, s))) return st;
    if ((st = bscale_host<float, double>(E, Bf.tmp, b, isb, E.act, s))) return st;
    if ((st = bprecond<float>(E, live, Bf.tmp, Bf.c, s))) return st;
    const float* cc = Bf.c;
    if ((st = bmdot<float>(E, &cc, 0, Bf.c, true, E.act, s))) return st;
    if ((st = sync_hv(E, 1))) return st;
    for (int i : live) nb[i] = sb[i] * std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv]));
  }
  std::vector<double> eta(E.B, 1.0);
  for (int it = 0; it <= o.max_refinements && !live.empty(); ++it) {
    if ((st = upload_mask(E, E.act, live, s))) return st;
    // r64 = b - A u (FP64, batched)
    if ((st = bapply<double>(E, K, u, E.r64, s))) return st;
    for (int i : live) info[i].applies_fp64++;
    if ((st = k_residual<double>(E.r64, b, (size_t)n, s))) return st;
    const double* rr = E.r64;
    if ((st = bmdot<double>(E, &rr, 0, E.r64, true, E.act, s))) return st;
    if ((st = sync_hv(E, 1))) return st;
    std::vector<double> sr(E.B, 0.0), isr(E.B, 0.0);
    std::vector<int> go;
    for (int i : live) {
      sr[i] = std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv]));
      if (!std::isfinite(sr[i])) { set_error("non-finite residual in a batched solve"); return CHEB_ERR_NONFINITE; }
      if (sr[i] == 0.0) { eta[i] = 0.0; info[i].status = CHEB_OK; continue; }
      isr[i] = 1.0 / sr[i];
      go.push_back(i);
    }
    live = go;
    if (live.empty()) break;
    if ((st = upload_mask(E, E.act, live, s))) return st;
    if ((st = bscale_host<float, double>(E, Bf.tmp, E.r64, isr, E.act, s))) return st;
    if ((st = bprecond<float>(E, live, Bf.tmp, Bf.c, s))) return st;
    const float* cc = Bf.c;
    if ((st = bmdot<float>(E, &cc, 0, Bf.c, true, E.act, s))) return st;
    if ((st = sync_hv(E, 1))) return st;
    std::vector<double> tol(E.B, 0.0);
    go.clear();
    for (int i : live) {
      const double cn = std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv]));
      eta[i] = sr[i] * cn / nb[i];
      info[i].rel_residual = eta[i];
      if (eta[i] <= o.rtol || sr[i] * cn <= o.atol) { info[i].status = CHEB_OK; continue; }
      if (it == o.max_refinements || info[i].iterations >= o.maxiter) { info[i].status = CHEB_ERR_NOT_CONVERGED; continue; }
      tol[i] = std::max(o.inner_rtol, 0.5 * o.rtol / eta[i]) * cn;  // as the single solve
      go.push_back(i);
    }
    live = go;
    if (live.empty()) break;
    int inner_max = o.inner_maxiter;
    for (int i : live) inner_max = std::min(inner_max, o.maxiter - info[i].iterations);
    BStats si;
    si.init(E.B);
    if ((st = blgmres<float>(E, live, o.restart, o.augment, std::max(1, inner_max), tol, Bf.K, Bf.c, Bf.x, true, si)))
      return st;
    for (int i : live) {
      info[i].iterations += si.iterations[i];
      info[i].cycles += si.cycles[i];
      info[i].applies_fp32 += si.applies[i];
      info[i].refinements++;
      info[i].host_syncs += si.syncs;
      info[i].rel_residual_inner = si.resid[i];
    }
    // u += sr_i x_i
    if ((st = upload_mask(E, E.act, live, s))) return st;
    CHEB_CUDA(cudaMemcpyAsync(E.fac, sr.data(), sizeof(double) * E.B, cudaMemcpyHostToDevice, s));
    baxpy64_kernel<float><<<E.bb.nblk, 256, 0, s>>>(E.bb, u, Bf.x, E.fac, E.act);
    CHEB_LAUNCH_CHECK("baxpy64_kernel");
  }
  CHEB_CUDA(cudaStreamSynchronize(s));
  return CHEB_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// entry points used by cheb_solve_batched / cheb_picard_batched (solve.cu)
// ---------------------------------------------------------------------------
bool lockstep_ok(int count, const cheb_plan* plans, const cheb_solve_opts& o) {
  if (count < 1 || o.formulation != CHEB_FORM_REPLACE || o.restart + o.augment + 1 > kMaxVecs) return false;
  if (o.reorth) return false;
  for (int i = 0; i < count; ++i) {
    const cheb_plan_s* p = plans[i];
    if (!p || p->dim != plans[0]->dim || p->device != plans[0]->device) return false;
    for (int a = 0; a < p->dim; ++a)
      if (!p->ax[a].dense_ok) return false;
    bool dir = false;
    for (int f = 0; f < 2 * p->dim; ++f) dir |= p->bc[f] == CHEB_DIRICHLET;
    if (!dir) return false;
  }
  return true;
}

// Packs the instances' fields into the batch vectors, solves (Picard when
// picard), unpacks u.  Per-instance infos; returns the worst status.
int lockstep_solve(int count, const cheb_plan* plans, const double* const* K, const double* const* b,
                   double* const* u, const cheb_solve_opts& o, cheb_solve_info* infos, bool picard, double beta,
                   double omega, double ptol, int pmaxit, int* piters) {
  const double t0 = now_s();
  Engine E;
  // the instances' preconditioners read their mask slot during the call
  struct Unmask {
    Engine* e;
    ~Unmask() {
      for (Fdm* f : e->fdm)
        if (f) f->active = nullptr;
    }
  } unmask{&E};
  int st;
  if (!pmat_ok(o)) return CHEB_ERR_ARG;
  if ((st = engine_setup(E, count, plans, o.precond))) return st;
  for (int i = 0; i < count; ++i)
    if (E.fdm[i]) {
      E.fdm[i]->active = E.act + i;
      E.fdm[i]->tf32_mats = o.precond_matrices == CHEB_PMAT_TF32;
    }
  const size_t tb = sizeof(double) * (size_t)E.total;
  double *Kb = nullptr, *bb = nullptr, *ub = nullptr, *Kp = nullptr, *u0 = nullptr, *G[3] = {nullptr, nullptr, nullptr};
  struct Free {
    std::vector<double*> v;
    ~Free() { for (double* p : v) if (p) cudaFree(p); }
  } fr;
  auto alloc = [&](double** p) -> int {
    CHEB_CUDA(cudaMalloc(p, tb));
    fr.v.push_back(*p);
    CHEB_CUDA(cudaMemsetAsync(*p, 0, tb, E.s));
    return CHEB_OK;
  };
  if ((st = alloc(&Kb)) || (st = alloc(&bb)) || (st = alloc(&ub))) return st;
  // the callers' arrays are on their plans' streams: finish that work first
  for (int i = 0; i < count; ++i) CHEB_CUDA(cudaStreamSynchronize(plans[i]->stream));
  for (int i = 0; i < count; ++i) {
    const size_t bytes = sizeof(double) * (size_t)E.len[i];
    CHEB_CUDA(cudaMemcpyAsync(Kb + E.off[i], K[i], bytes, cudaMemcpyDeviceToDevice, E.s));
    CHEB_CUDA(cudaMemcpyAsync(bb + E.off[i], b[i], bytes, cudaMemcpyDeviceToDevice, E.s));
    CHEB_CUDA(cudaMemcpyAsync(ub + E.off[i], u[i], bytes, cudaMemcpyDeviceToDevice, E.s));
  }
  std::vector<cheb_solve_info> info(count);
  for (auto& x : info) std::memset(&x, 0, sizeof(x));
  std::vector<int> live;
  for (int i = 0; i < count; ++i) live.push_back(i);
  std::vector<int> rc(count, CHEB_OK);
  if (!picard) {
    if ((st = bsolve(E, live, o, Kb, bb, ub, info, false))) return st;
    for (int i = 0; i < count; ++i) rc[i] = info[i].status;
  } else {
    if ((st = alloc(&Kp)) || (st = alloc(&u0))) return st;
    for (int a = 0; a < E.dim; ++a)
      if ((st = alloc(&G[a]))) return st;
    std::vector<int> its(count, 0);
    std::vector<cheb_solve_info> tot(count);
    for (auto& x : tot) std::memset(&x, 0, sizeof(x));
    for (int i = 0; i < count; ++i) rc[i] = CHEB_ERR_NOT_CONVERGED;
    for (int m = 1; m <= pmaxit && !live.empty(); ++m) {
      if ((st = upload_mask(E, E.act, live, E.s))) return st;
      // K^m = K0 (1 + beta |grad u|^2): batched derivative passes (FP64)
      for (int a = 0; a < E.dim; ++a)
        if ((st = bpass<double>(E, a, kDeriv, nullptr, ub, G[a], E.s))) return st;
      bpicard_k_kernel<<<grid1(E.total), 256, 0, E.s>>>(Kb, G[0], E.dim > 1 ? G[1] : nullptr,
                                                       E.dim > 2 ? G[2] : nullptr, beta, Kp, E.total);
      CHEB_LAUNCH_CHECK("bpicard_k_kernel");
      CHEB_CUDA(cudaMemcpyAsync(u0, ub, tb, cudaMemcpyDeviceToDevice, E.s));
      std::vector<cheb_solve_info> li(count);
      for (auto& x : li) std::memset(&x, 0, sizeof(x));
      // kref frozen after the first Picard step: captured step graphs stay valid
      if ((st = bsolve(E, live, o, Kp, bb, ub, li, m > 1))) return st;
      for (int i : live) {
        tot[i].iterations += li[i].iterations;
        tot[i].cycles += li[i].cycles;
        tot[i].refinements += li[i].refinements;
        tot[i].applies_fp64 += li[i].applies_fp64;
        tot[i].applies_fp32 += li[i].applies_fp32;
        tot[i].host_syncs += li[i].host_syncs;
        tot[i].rel_residual = li[i].rel_residual;
        tot[i].rel_residual_inner = li[i].rel_residual_inner;
        tot[i].kref = li[i].kref;
        its[i] = m;
      }
      if (omega != 1.0) {
        brelax_kernel<<<grid1(E.total), 256, 0, E.s>>>(ub, u0, omega, E.total);
        CHEB_LAUNCH_CHECK("brelax_kernel");
      }
      if ((st = upload_mask(E, E.act, live, E.s))) return st;
      bdiff_kernel<<<E.bb.nblk, kBThreads, 0, E.s>>>(E.bb, ub, u0, E.act, E.part, E.counter, E.dv);
      CHEB_LAUNCH_CHECK("bdiff_kernel");
      if ((st = sync_hv(E, 2))) return st;
      std::vector<int> next;
      for (int i : live) {
        const double dn = std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv]));
        const double un = std::sqrt(std::max(0.0, E.hv[(size_t)i * kDv + 1]));
        const double d = un > 0 ? dn / un : dn;
        if (!std::isfinite(d)) { set_error("non-finite Picard update in a batched solve"); return CHEB_ERR_NONFINITE; }
        if (li[i].status < 0) { rc[i] = li[i].status; continue; }
        if (d <= ptol) { rc[i] = CHEB_OK; continue; }
        next.push_back(i);
      }
      live = next;
    }
    info = tot;
    if (piters)
      for (int i = 0; i < count; ++i) piters[i] = its[i];
  }
  for (int i = 0; i < count; ++i)
    CHEB_CUDA(cudaMemcpyAsync(u[i], ub + E.off[i], sizeof(double) * (size_t)E.len[i], cudaMemcpyDeviceToDevice, E.s));
  CHEB_CUDA(cudaStreamSynchronize(E.s));
  const double dt = now_s() - t0;
  int worst = CHEB_OK;
  for (int i = 0; i < count; ++i) {
    info[i].status = rc[i];
    info[i].seconds = dt;
    info[i].graph_captures = E.captures;
    if (infos) infos[i] = info[i];
    if (rc[i] < 0 && (worst >= 0 || rc[i] < worst)) worst = rc[i];
    else if (worst == CHEB_OK && rc[i] > 0) worst = rc[i];
  }
  return worst;
}

}  // namespace cheb
