// Solver drivers: LGMRES(m, k) on the left-preconditioned collocation system
// (the Krylov solver named in Alg. 2; Baker, Jessup & Manteuffel 2005: m new
// Krylov directions plus k error-approximation vectors carried between
// restart cycles), and the mixed-precision form: FP32 inner LGMRES cycles
// inside an FP64 iterative-refinement loop.
//
// Arnoldi step j (classical Gram-Schmidt, optionally twice):
//   w = M^{-1} A v_j           (line passes + preconditioner)
//   h = V_j^T w                (one fused multi-dot kernel, deterministic)
//   w -= V_j h, ||w||          (one fused multi-axpy kernel with the norm)
//   v_{j+1} = w / ||w||
// The Hessenberg least-squares problem (Givens rotations) is solved on the
// host in FP64 after one stream synchronisation per step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <thread>
#include <vector>

#include "device.cuh"
#include "fdm.h"
#include "hess.cuh"
#include "umma.h"
#include "krylov.h"
#include "prolong.h"

namespace cheb {

// Captured Arnoldi cycles, one per cycle shape (number of Krylov steps).
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  long long nkernels = 0;  // kernel launches captured in the graph
  int m_eff = -1;
  const void* K = nullptr;
  double kref = 0.0;
  int precond = -1, pmat = -1, reorth = -1, transpose = -1, m = -1, k = -1;
};

template <typename T>
struct KrylovBufs {
  int nvec = 0;        // allocated basis vectors
  int kaug = 0;        // allocated augmentation pairs
  size_t ld = 0;       // vector stride: n rounded up to 64 elements (256-byte aligned vectors)
  T* V = nullptr;      // nvec x ld
  T* Z = nullptr;      // kaug x ld (error approximations)
  T* BZ = nullptr;     // kaug x ld (M^{-1} A z)
  T* tmp = nullptr;    // n
  T* x = nullptr;      // n (inner solution)
  T* c = nullptr;      // n (inner right-hand side)
  T* K = nullptr;      // n (conductivity in this precision)
  CycleGraph graphs[kMaxVecs];
};

struct Workspace {
  size_t n = 0;
  ReduceScratch rs;
  double* dscal = nullptr;    // device scalars (dots, norms): kMaxVecs + 8
  double* hscal = nullptr;    // pinned host mirror
  KrylovBufs<double> k64;
  KrylovBufs<float> k32;
  double* r64 = nullptr;      // FP64 residual
  double* pro[3] = {nullptr, nullptr, nullptr};  // prolongation scratch (2) + prolonged copy
  double* adj[3] = {nullptr, nullptr, nullptr};  // gradient accumulation / Picard temporaries
  double* dhess = nullptr;    // device Hessenberg / Givens state of graph cycles
  double* hhess = nullptr;    // pinned mirror
  int* dorder = nullptr;      // augmentation slot order (device) and pinned mirror
  int* horder = nullptr;
  cudaStream_t gstream = nullptr;  // private stream for graph capture
  double* lvl[3] = {nullptr, nullptr, nullptr};  // recomputed coarse level: K, b, u (hierarchy from fine data)
  double* picK = nullptr;                         // Picard conductivity
  double* picU = nullptr;                         // Picard previous iterate
  Fdm fdm;
};

template <typename T> static KrylovBufs<T>& bufs(Workspace& w);
template <> KrylovBufs<double>& bufs<double>(Workspace& w) { return w.k64; }
template <> KrylovBufs<float>& bufs<float>(Workspace& w) { return w.k32; }

template <typename T>
static void free_bufs(KrylovBufs<T>& b) {
  cudaFree(b.V); cudaFree(b.Z); cudaFree(b.BZ); cudaFree(b.tmp); cudaFree(b.x); cudaFree(b.c); cudaFree(b.K);
  for (auto& g : b.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  b = KrylovBufs<T>();
}

void free_workspace(cheb_plan_s* p) {
  if (!p->ws) return;
  Workspace* w = p->ws;
  cudaFree(w->rs.part); cudaFree(w->rs.counter); cudaFree(w->dscal); cudaFreeHost(w->hscal);
  free_bufs(w->k64); free_bufs(w->k32);
  cudaFree(w->r64);
  for (int i = 0; i < 3; ++i) { cudaFree(w->pro[i]); cudaFree(w->adj[i]); }
  cudaFree(w->picK);
  cudaFree(w->picU);
  for (int i = 0; i < 3; ++i) cudaFree(w->lvl[i]);
  cudaFree(w->dhess);
  cudaFreeHost(w->hhess);
  cudaFree(w->dorder);
  cudaFreeHost(w->horder);
  if (w->gstream) cudaStreamDestroy(w->gstream);
  fdm_free(w->fdm);
  delete w;
  p->ws = nullptr;
}

static int ensure_ws(cheb_plan_s* p) {
  if (p->ws) return CHEB_OK;
  Workspace* w = new Workspace();
  p->ws = w;
  w->n = p->size();
  CHEB_CUDA(cudaMalloc(&w->rs.part, sizeof(double) * (kMaxVecs + 1) * kRedBlocks));
  CHEB_CUDA(cudaMalloc(&w->rs.counter, sizeof(unsigned)));
  CHEB_CUDA(cudaMemset(w->rs.counter, 0, sizeof(unsigned)));
  CHEB_CUDA(cudaMalloc(&w->dscal, sizeof(double) * (kMaxVecs + 8)));
  CHEB_CUDA(cudaMallocHost(&w->hscal, sizeof(double) * (kMaxVecs + 8)));
  return CHEB_OK;
}

template <typename T>
static int ensure_bufs(Workspace& w, int nvec, int kaug) {
  KrylovBufs<T>& b = bufs<T>(w);
  const size_t n = w.n;
  b.ld = (n + 63) / 64 * 64;
  if (b.nvec < nvec) {
    cudaFree(b.V);
    b.V = nullptr;
    CHEB_CUDA(cudaMalloc(&b.V, sizeof(T) * b.ld * nvec));
    b.nvec = nvec;
  }
  if (b.kaug < kaug) {
    cudaFree(b.Z); cudaFree(b.BZ);
    b.Z = b.BZ = nullptr;
    CHEB_CUDA(cudaMalloc(&b.Z, sizeof(T) * b.ld * kaug));
    CHEB_CUDA(cudaMalloc(&b.BZ, sizeof(T) * b.ld * kaug));
    b.kaug = kaug;
  }
  if (!b.tmp) {
    CHEB_CUDA(cudaMalloc(&b.tmp, sizeof(T) * n));
    CHEB_CUDA(cudaMalloc(&b.x, sizeof(T) * n));
    CHEB_CUDA(cudaMalloc(&b.c, sizeof(T) * n));
    CHEB_CUDA(cudaMalloc(&b.K, sizeof(T) * n));
  }
  return CHEB_OK;
}

static int sync_read(Workspace& w, int cnt, cudaStream_t s) {
  CHEB_CUDA(cudaMemcpyAsync(w.hscal, w.dscal, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
  CHEB_CUDA(cudaStreamSynchronize(s));
  return CHEB_OK;
}

// Settings of one LGMRES run.
struct LgOpts {
  int m = 30, k = 3, maxiter = 1000;
  bool reorth = false;
  bool transpose = false;  // solve with A^T and M^{-T} (adjoint)
  bool use_graph = false;  // run Arnoldi cycles as captured CUDA graphs
  int precond = CHEB_PRECOND_FDM;
  int pmat = CHEB_PMAT_TF32;  // FP32 preconditioner matrices (part of the graph key)
  double kref = 1.0;
  double tol_abs = 0.0;  // stop when ||c - B x|| <= tol_abs
  const void* jac[3] = {nullptr, nullptr, nullptr};  // Newton: operator J (C_a fields, type T)
  bool elim = false;              // elimination formulation: B v = P_int A(E_0 v) (FP64)
  const void* elim_zero = nullptr;  // a zero field (homogeneous boundary data)
};

__global__ void mask_interior_kernel(Geom g, const double* __restrict__ x, double* __restrict__ y);

// Augmentation vectors carried from one LGMRES call to the next on the same
// operator (the FP32 inner solves of one refinement loop): their count and
// the next slot of the circular Z / BZ store.
struct LgCarry {
  int naug = 0, next_slot = 0;
};

struct LgStats {
  int iterations = 0, cycles = 0, applies = 0, captures = 0;
  int syncs = 0;      // host synchronisations of the Arnoldi cycles
  int overshoot = 0;  // Arnoldi steps run past the converged one (discarded)
  double resid = 0.0;  // last true preconditioned residual norm
  bool converged = false;
};

// out = B v = M^{-1} A v (tmp holds A v)
template <typename T> struct Cat;
template <> struct Cat<double> { static constexpr int apply = kProfApply64, prec = kProfPrec64, orth = kProfOrth64; };
template <> struct Cat<float> { static constexpr int apply = kProfApply32, prec = kProfPrec32, orth = kProfOrth32; };

template <typename T>
static int op_B(cheb_plan_s* p, Workspace& w, const LgOpts& o, const T* K, const T* v, T* out, T* tmp,
                cudaStream_t s) {
  int st;
  if constexpr (sizeof(T) == 8) {
    if (o.elim) {
      // B v = [M_int^{-1}] P_int A(E_0 v): boundary values of v from its
      // interior by the elimination with zero data, the operator, interior rows
      const size_t n = p->size();
      const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 8));
      prof_begin(kProfOther, s);
      CHEB_CUDA(cudaMemcpyAsync(tmp, v, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
      if ((st = fdm_fill_boundary<T>(p, w.fdm, (const T*)o.elim_zero, tmp, s))) return st;
      prof_end(kProfOther, s);
      prof_begin(Cat<T>::apply, s);
      if ((st = launch_apply<T>(p, K, tmp, out, s))) return st;
      prof_end(Cat<T>::apply, s);
      mask_interior_kernel<<<blocks, 256, 0, s>>>(p->geom(), out, out);
      CHEB_LAUNCH_CHECK("mask_interior_kernel");
      if (o.precond != CHEB_PRECOND_FDM) return CHEB_OK;
      prof_begin(Cat<T>::prec, s);
      if ((st = fdm_apply<T>(p, w.fdm, o.kref, out, tmp, s))) return st;
      prof_end(Cat<T>::prec, s);
      mask_interior_kernel<<<blocks, 256, 0, s>>>(p->geom(), tmp, out);
      CHEB_LAUNCH_CHECK("mask_interior_kernel");
      return CHEB_OK;
    }
  }
  prof_begin(Cat<T>::apply, s);
  T* dst = o.precond == CHEB_PRECOND_FDM ? tmp : out;
  if (o.jac[0]) {
    const T* C[3] = {(const T*)o.jac[0], (const T*)o.jac[1], (const T*)o.jac[2]};
    st = launch_jacobian<T>(p, K, C, v, dst, s);
  } else {
    st = o.transpose ? launch_adjoint_apply<T>(p, K, v, dst, s) : launch_apply<T>(p, K, v, dst, s);
  }
  prof_end(Cat<T>::apply, s);
  if (st || o.precond != CHEB_PRECOND_FDM) return st;
  prof_begin(Cat<T>::prec, s);
  st = o.transpose ? fdm_apply_t<T>(p, w.fdm, o.kref, tmp, out, s)
                   : fdm_apply<T>(p, w.fdm, o.kref, tmp, out, s);
  prof_end(Cat<T>::prec, s);
  return st;
}

// Hessenberg column and Givens rotation of step j on the device (hess.cuh)
__global__ void hcol_kernel(double* hess, HessLayout L, int j, int pass, const double* __restrict__ dv) {
  hess_column(hess, L, j, pass, dv);
}
__global__ void givens_kernel(double* hess, HessLayout L, int j, const double* __restrict__ norm2) {
  if (threadIdx.x == 0) hess_givens(hess, L, j, *norm2);
}

// w = BZ[order[q]] (augmentation step q of a cycle; vectors ld apart)
template <typename T>
__global__ void copy_slot_kernel(T* __restrict__ w, const T* __restrict__ BZ, const int* __restrict__ order,
                                 int q, size_t n, size_t ld) {
  const T* src = BZ + (size_t)order[q] * ld;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    w[c] = src[c];
}

static int ensure_hess(Workspace& w) {
  if (w.dhess) return CHEB_OK;
  HessLayout Lmax{kMaxVecs};
  CHEB_CUDA(cudaMalloc(&w.dhess, sizeof(double) * Lmax.total()));
  CHEB_CUDA(cudaMallocHost(&w.hhess, sizeof(double) * Lmax.total()));
  CHEB_CUDA(cudaMalloc(&w.dorder, sizeof(int) * kMaxVecs));
  CHEB_CUDA(cudaMallocHost(&w.horder, sizeof(int) * kMaxVecs));
  return CHEB_OK;
}

// One Arnoldi cycle as a CUDA graph: captured once per cycle shape and
// operator (K, kref, options), replayed afterwards.  The host reads the
// Hessenberg state once at the end and keeps the steps up to the first one
// whose residual estimate meets the tolerance (later steps only extend the
// basis and are ignored).
template <typename T>
static int graph_cycle(cheb_plan_s* p, Workspace& w, const LgOpts& o, const T* K, int m_eff, int naug,
                       int next_slot, double beta, int steps_max, int nbasis,
                       std::vector<double>& H, std::vector<double>& Hr, std::vector<double>& g,
                       LgStats& stt, int& steps, cudaStream_t s) {
  const size_t n = w.n;
  KrylovBufs<T>& B = bufs<T>(w);
  const int kk = o.k;
  HessLayout L{nbasis};
  int st0;
  if ((st0 = ensure_hess(w))) return st0;
  // per-cycle inputs: g = (beta, 0, ...), augmentation order (oldest first)
  std::fill(w.hhess, w.hhess + L.total(), 0.0);
  w.hhess[L.g()] = beta;
  for (int q = 0; q < naug; ++q) w.horder[q] = (next_slot - naug + q + 4 * kk) % std::max(1, kk);
  CHEB_CUDA(cudaMemcpyAsync(w.dhess, w.hhess, sizeof(double) * L.total(), cudaMemcpyHostToDevice, s));
  CHEB_CUDA(cudaMemcpyAsync(w.dorder, w.horder, sizeof(int) * std::max(1, naug), cudaMemcpyHostToDevice, s));
  CycleGraph& cg = B.graphs[m_eff];
  const bool match = cg.exec && cg.m_eff == m_eff && cg.K == (const void*)K && cg.kref == o.kref &&
                     cg.precond == o.precond && cg.pmat == o.pmat && cg.reorth == (int)o.reorth &&
                     cg.transpose == (int)o.transpose &&
                     cg.m == o.m && cg.k == o.k;
  if (!match) {
    if (cg.exec) { cudaGraphExecDestroy(cg.exec); cg.exec = nullptr; }
    double* dv = w.dscal;
    auto Vp = [&](int i) { return B.V + (size_t)i * B.ld; };
    // one uncaptured application first: lazy workspace allocation and kernel
    // attributes happen outside the capture
    {
      int st0 = op_B<T>(p, w, o, K, Vp(0), Vp(1), B.tmp, s);
      if (st0) return st0;
      CHEB_CUDA(cudaStreamSynchronize(s));
    }
    // capture on a private stream (the legacy stream cannot be captured); the
    // graph is launched on the plan's stream afterwards
    if (!w.gstream) CHEB_CUDA(cudaStreamCreateWithFlags(&w.gstream, cudaStreamNonBlocking));
    cudaStream_t cs = w.gstream;
    const long long l0 = thread_launches();
    CHEB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int st = CHEB_OK;
    for (int j = 0; j < steps_max && st == CHEB_OK; ++j) {
      T* wv = Vp(j + 1);
      if (j < m_eff) {
        st = op_B<T>(p, w, o, K, Vp(j), wv, B.tmp, cs);
      } else {
        copy_slot_kernel<T><<<(int)std::min<size_t>((n + 255) / 256, 148 * 8), 256, 0, cs>>>(wv, B.BZ, w.dorder,
                                                                                              j - m_eff, n, B.ld);
        count_launch();
      }
      const T* src[kMaxVecs];
      for (int i = 0; i <= j; ++i) src[i] = Vp(i);
      for (int pass = 0; pass < (o.reorth ? 2 : 1) && st == CHEB_OK; ++pass) {
        if ((st = k_mdot<T>(w.rs, src, j + 1, wv, n, false, dv, cs))) break;
        if ((st = k_maxpy_dev<T>(w.rs, src, dv, -1.0, j + 1, 1.0, wv, n, dv + kMaxVecs + 1, cs))) break;
        hcol_kernel<<<1, 64, 0, cs>>>(w.dhess, L, j, pass, dv);
        count_launch();
      }
      if (st) break;
      if ((st = k_scale_inv_norm<T>(wv, dv + kMaxVecs + 1, n, cs))) break;
      givens_kernel<<<1, 32, 0, cs>>>(w.dhess, L, j, dv + kMaxVecs + 1);
      count_launch();
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (st) { if (graph) cudaGraphDestroy(graph); return st; }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&cg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { cg.exec = nullptr; return cuda_fail(ce, "cudaGraphInstantiate"); }
    cg.m_eff = m_eff; cg.K = K; cg.kref = o.kref; cg.precond = o.precond; cg.pmat = o.pmat; cg.reorth = o.reorth;
    cg.transpose = o.transpose; cg.m = o.m; cg.k = o.k;
    cg.nkernels = thread_launches() - l0;
    add_launches(-cg.nkernels);  // recorded, not run: counted at each replay
    stt.captures++;
  }
  prof_begin(kProfOther, s);
  CHEB_CUDA(cudaGraphLaunch(cg.exec, s));
  prof_end(kProfOther, s);
  add_launches(cg.nkernels);
  CHEB_CUDA(cudaMemcpyAsync(w.hhess, w.dhess, sizeof(double) * L.total(), cudaMemcpyDeviceToHost, s));
  CHEB_CUDA(cudaStreamSynchronize(s));
  const double* hh = w.hhess;
  steps = steps_max;
  for (int j = 0; j < steps_max; ++j) {
    const double r = hh[L.res() + j];
    if (!std::isfinite(r) || r <= o.tol_abs || stt.iterations + j + 1 >= o.maxiter) { steps = j + 1; break; }
  }
  if (!std::isfinite(hh[L.res() + steps - 1])) { set_error("non-finite Arnoldi residual"); return CHEB_ERR_NONFINITE; }
  stt.syncs++;
  stt.overshoot += steps_max - steps;
  stt.iterations += steps;
  stt.applies += std::min(steps, m_eff);
  for (size_t i = 0; i < (size_t)(nbasis + 1) * nbasis; ++i) {
    H[i] = hh[L.H() + i];
    Hr[i] = hh[L.R() + i];
  }
  for (int i = 0; i <= nbasis; ++i) g[i] = hh[L.g() + i];
  // g must be the rotated right-hand side after `steps` rotations: recompute it
  // from the rotations (later rotations only touch entries beyond `steps`)
  std::fill(g.begin(), g.end(), 0.0);
  g[0] = beta;
  for (int j = 0; j < steps; ++j) {
    const double c = hh[L.cs() + j], sn = hh[L.sn() + j];
    g[j + 1] = -sn * g[j];
    g[j] = c * g[j];
  }
  return CHEB_OK;
}

// LGMRES on B x = c (B = M^{-1} A), x in/out.  Returns CHEB_OK when
// converged, CHEB_ERR_NOT_CONVERGED at maxiter, or an error.
template <typename T>
static int lgmres(cheb_plan_s* p, Workspace& w, const LgOpts& o, const T* K, const T* c, T* x,
                  bool x_is_zero, LgStats& stt, cudaStream_t s, LgCarry* carry = nullptr) {
  const size_t n = w.n;
  const int m = o.m, kk = o.k;
  const int nbasis = m + kk + 1;
  int st;
  if ((st = ensure_bufs<T>(w, nbasis, std::max(1, kk)))) return st;
  KrylovBufs<T>& B = bufs<T>(w);
  auto Vp = [&](int i) { return B.V + (size_t)i * B.ld; };
  auto Zp = [&](int i) { return B.Z + (size_t)i * B.ld; };
  auto BZp = [&](int i) { return B.BZ + (size_t)i * B.ld; };
  int naug = 0, next_slot = 0;
  if (carry && kk > 0) {
    naug = std::min(carry->naug, kk);
    next_slot = carry->next_slot % kk;
  }
  // record the augmentation state on every return
  struct SaveCarry {
    LgCarry* c;
    int* naug;
    int* next;
    ~SaveCarry() {
      if (c) { c->naug = *naug; c->next_slot = *next; }
    }
  } save_carry{carry, &naug, &next_slot};
  std::vector<double> H((size_t)(nbasis + 1) * nbasis), Hr((size_t)(nbasis + 1) * nbasis);
  std::vector<double> cs(nbasis), sn(nbasis), g(nbasis + 1), y(nbasis);
  double* dv = w.dscal;
  double* hv = w.hscal;
  bool zero = x_is_zero;
  bool last_full = false;  // previous cycle ran all its steps (graph replay pays off)
  double lg_rate = 0.0;     // observed residual reduction per Arnoldi step
  stt = LgStats();
  while (true) {
    // ---- residual r = c - B x into V[0]
    if (zero) {
      prof_begin(kProfOther, s);
      if ((st = k_scale<T>(Vp(0), c, 1.0, n, s))) return st;
      prof_end(kProfOther, s);
    } else {
      if ((st = op_B<T>(p, w, o, K, x, Vp(0), B.tmp, s))) return st;
      stt.applies++;
      prof_begin(kProfOther, s);
      if ((st = k_residual<T>(Vp(0), c, n, s))) return st;
      prof_end(kProfOther, s);
    }
    const T* v0 = Vp(0);
    prof_begin(Cat<T>::orth, s);
    if ((st = k_mdot<T>(w.rs, &v0, 0, Vp(0), n, true, dv, s))) return st;
    prof_end(Cat<T>::orth, s);
    if ((st = sync_read(w, 1, s))) return st;
    stt.syncs++;
    const double beta = std::sqrt(hv[0]);
    stt.resid = beta;
    if (!std::isfinite(beta)) { set_error("non-finite residual"); return CHEB_ERR_NONFINITE; }
    if (beta <= o.tol_abs) { stt.converged = true; return CHEB_OK; }
    if (stt.iterations >= o.maxiter) return CHEB_ERR_NOT_CONVERGED;
    prof_begin(Cat<T>::orth, s);
    if ((st = k_scale<T>(Vp(0), Vp(0), 1.0 / beta, n, s))) return st;
    prof_end(Cat<T>::orth, s);
    stt.cycles++;
    // ---- Arnoldi: first m_eff Krylov directions, then the augmentation vectors
    const int m_eff = m + (kk - naug);
    const int steps_max = m_eff + naug;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int steps = 0;
    const bool graph = o.use_graph && last_full;
    if (graph) {
      if ((st = graph_cycle<T>(p, w, o, K, m_eff, naug, next_slot, beta, steps_max, nbasis, H, Hr, g,
                               stt, steps, s)))
        return st;
    }
    if (!graph) {
      // Arnoldi steps with the Hessenberg column and its Givens rotation on
      // the device (hcol_kernel, givens_kernel): nothing returns to the host
      // per step.  The host reads the device state at checkpoints only: the
      // end of the cycle, and earlier when the residual estimates predict
      // convergence (from the reduction rate seen so far), so a cycle far
      // from the tolerance costs one synchronisation.  Steps run past the
      // first converged one are discarded (counted in stt.overshoot).
      if ((st = ensure_hess(w))) return st;
      HessLayout L{nbasis};
      const int budget = std::min(steps_max, std::max(1, o.maxiter - stt.iterations));
      std::fill(w.hhess, w.hhess + L.total(), 0.0);
      w.hhess[L.g()] = beta;
      CHEB_CUDA(cudaMemcpyAsync(w.dhess, w.hhess, sizeof(double) * L.total(), cudaMemcpyHostToDevice, s));
      // Arnoldi steps to go until r <= tol_abs at the observed rate (8 without one)
      auto predict = [&](double r) -> int {
        if (!(lg_rate > 0.0 && lg_rate < 1.0) || !(r > o.tol_abs)) return 8;
        const double k = std::ceil(std::log(o.tol_abs / r) / std::log(lg_rate));
        return (int)std::max(1.0, std::min(k, 1e6));
      };
      int next_check = std::min(budget, predict(beta));
      int checked = 0;  // steps already inspected on the host
      steps = -1;
      for (int j = 0; j < budget; ++j) {
        T* wv = Vp(j + 1);
        if (j < m_eff) {
          if ((st = op_B<T>(p, w, o, K, Vp(j), wv, B.tmp, s))) return st;
          stt.applies++;
        } else {
          const int a = (next_slot - naug + (j - m_eff) + 4 * kk) % kk;  // oldest first
          prof_begin(Cat<T>::orth, s);
          if ((st = k_scale<T>(wv, BZp(a), 1.0, n, s))) return st;
          prof_end(Cat<T>::orth, s);
        }
        const T* src[kMaxVecs];
        for (int i = 0; i <= j; ++i) src[i] = Vp(i);
        // classical Gram-Schmidt (twice if requested): h = V^T w, w -= V h, |w|^2
        prof_begin(Cat<T>::orth, s);
        for (int pass = 0; pass < (o.reorth ? 2 : 1); ++pass) {
          if ((st = k_mdot<T>(w.rs, src, j + 1, wv, n, false, dv, s))) return st;
          if ((st = k_maxpy_dev<T>(w.rs, src, dv, -1.0, j + 1, 1.0, wv, n, dv + kMaxVecs + 1, s))) return st;
          hcol_kernel<<<1, 64, 0, s>>>(w.dhess, L, j, pass, dv);
          CHEB_LAUNCH_CHECK("hcol_kernel");
        }
        if ((st = k_scale_inv_norm<T>(wv, dv + kMaxVecs + 1, n, s))) return st;
        givens_kernel<<<1, 32, 0, s>>>(w.dhess, L, j, dv + kMaxVecs + 1);
        CHEB_LAUNCH_CHECK("givens_kernel");
        prof_end(Cat<T>::orth, s);
        if (j + 1 < next_check && j + 1 < budget) continue;
        // ---- checkpoint: read the Hessenberg state
        CHEB_CUDA(cudaMemcpyAsync(w.hhess, w.dhess, sizeof(double) * L.total(), cudaMemcpyDeviceToHost, s));
        CHEB_CUDA(cudaStreamSynchronize(s));
        stt.syncs++;
        const double* hh = w.hhess;
        for (int i = checked; i <= j; ++i) {
          const double r = hh[L.res() + i];
          if (!std::isfinite(r)) { set_error("non-finite Arnoldi residual"); return CHEB_ERR_NONFINITE; }
          if (r <= o.tol_abs) { steps = i + 1; break; }
        }
        if (steps < 0 && j + 1 >= 2) {
          // reduction rate per step over the steps of this cycle so far
          const double r1 = hh[L.res() + j], r0 = j >= 4 ? hh[L.res() + j - 4] : beta;
          const int span = j >= 4 ? 4 : j + 1;
          if (r1 > 0.0 && r0 > 0.0 && r1 < r0) lg_rate = std::pow(r1 / r0, 1.0 / span);
        }
        checked = j + 1;
        if (steps >= 0) { stt.overshoot += j + 1 - steps; break; }
        if (j + 1 >= budget) { steps = j + 1; break; }
        next_check = std::min(budget, j + 1 + predict(hh[L.res() + j]));
      }
      const double* hh = w.hhess;
      for (size_t i = 0; i < (size_t)(nbasis + 1) * nbasis; ++i) {
        H[i] = hh[L.H() + i];
        Hr[i] = hh[L.R() + i];
      }
      // the rotated right-hand side after `steps` rotations (later steps of
      // the cycle only touched entries beyond it)
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      for (int j = 0; j < steps; ++j) {
        const double c = hh[L.cs() + j], sn = hh[L.sn() + j];
        g[j + 1] = -sn * g[j];
        g[j] = c * g[j];
      }
      stt.iterations += steps;
    }
    last_full = steps == steps_max && std::fabs(g[steps]) > o.tol_abs;
    // ---- least squares: R y = g
    for (int i = steps - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < steps; ++l) t -= Hr[(size_t)i * nbasis + l] * y[l];
      y[i] = Hr[(size_t)i * nbasis + i] != 0.0 ? t / Hr[(size_t)i * nbasis + i] : 0.0;
    }
    // ---- dx = W y into tmp (with its norm), x += dx
    prof_begin(kProfOther, s);
    {
      const T* src[kMaxVecs];
      double coef[kMaxVecs];
      for (int i = 0; i < steps; ++i) {
        if (i < m_eff) src[i] = Vp(i);
        else src[i] = Zp((next_slot - naug + (i - m_eff) + 4 * kk) % kk);
        coef[i] = y[i];
      }
      if ((st = k_maxpy<T>(w.rs, src, coef, steps, 0.0, B.tmp, n, dv + kMaxVecs + 1, s))) return st;
      const T* one[1] = {B.tmp};
      double cone[1] = {1.0};
      if (zero) {
        if ((st = k_scale<T>(x, B.tmp, 1.0, n, s))) return st;
      } else {
        if ((st = k_maxpy<T>(w.rs, one, cone, 1, 1.0, x, n, nullptr, s))) return st;
      }
      zero = false;
      prof_end(kProfOther, s);
      if (kk > 0) {
        if ((st = sync_read(w, kMaxVecs + 2, s))) return st;
        stt.syncs++;
        const double dxn = std::sqrt(std::max(0.0, hv[kMaxVecs + 1]));
        if (dxn > 0) {
          // store z = dx/|dx| and B z = V Hbar y / |dx| (linearity: B W = V Hbar)
          const int slot = next_slot;
          prof_begin(kProfOther, s);
          if ((st = k_scale<T>(Zp(slot), B.tmp, 1.0 / dxn, n, s))) return st;
          prof_end(kProfOther, s);
          double hy[kMaxVecs];
          const T* vs[kMaxVecs];
          for (int i = 0; i <= steps; ++i) {
            double t = 0.0;
            for (int l = 0; l < steps; ++l)
              if (i <= l + 1) t += H[(size_t)i * nbasis + l] * y[l];
            hy[i] = t / dxn;
            vs[i] = Vp(i);
          }
          prof_begin(kProfOther, s);
          if ((st = k_maxpy<T>(w.rs, vs, hy, steps + 1, 0.0, BZp(slot), n, nullptr, s))) return st;
          prof_end(kProfOther, s);
          next_slot = (next_slot + 1) % kk;
          naug = std::min(naug + 1, kk);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// drivers
// ---------------------------------------------------------------------------
static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void default_opts(cheb_solve_opts& o) {
  std::memset(&o, 0, sizeof(o));
  o.mode = CHEB_SOLVE_MIXED;
  o.rtol = 1e-12;
  o.restart = 30;
  o.augment = 3;
  o.maxiter = 2000;
  o.inner_rtol = 1e-4;
  o.inner_maxiter = 400;
  o.max_refinements = 30;
  o.reorth = 0;
  o.precond = CHEB_PRECOND_FDM;
  o.kref = 0.0;
  o.use_graph = 0;
  o.recycle = 0;
  o.formulation = CHEB_FORM_REPLACE;
  o.coarse_rtol = 0.0;
  o.batch_mode = CHEB_BATCH_AUTO;
  o.precond_matrices = CHEB_PMAT_TF32;
}

// lockstep batch engine (batch.cu)
bool lockstep_ok(int count, const cheb_plan* plans, const cheb_solve_opts& o);
int lockstep_solve(int count, const cheb_plan* plans, const double* const* K, const double* const* b,
                   double* const* u, const cheb_solve_opts& o, cheb_solve_info* infos, bool picard, double beta,
                   double omega, double ptol, int pmaxit, int* piters);

// plan-level helpers of the lockstep batch engine (batch.cu)
int plan_fdm(cheb_plan_s* p, Fdm** f) {
  int st;
  if ((st = ensure_ws(p))) return st;
  if ((st = fdm_setup(p, p->ws->fdm))) return st;
  *f = &p->ws->fdm;
  return CHEB_OK;
}

// geometric mean of K over the plan's grid, computed on stream s (synchronises s)
int plan_kref(cheb_plan_s* p, const double* K, double* kref, cudaStream_t s) {
  int st;
  if ((st = ensure_ws(p))) return st;
  Workspace& w = *p->ws;
  if ((st = k_sum_log(w.rs, K, w.n, w.dscal, s))) return st;
  if ((st = sync_read(w, 1, s))) return st;
  *kref = std::exp(w.hscal[0] / (double)w.n);
  return CHEB_OK;
}

bool pmat_ok(const cheb_solve_opts& o) {
  if (o.precond_matrices == CHEB_PMAT_TF32 || o.precond_matrices == CHEB_PMAT_FP32) return true;
  set_error("precond_matrices must be CHEB_PMAT_TF32 or CHEB_PMAT_FP32");
  return false;
}

void resolve_opts(const cheb_solve_opts* in, cheb_solve_opts* out) {
  if (in) *out = *in;
  else default_opts(*out);
}

static double norm2_dev(Workspace& w, const double* x, cudaStream_t s, int* st) {
  const double* src[1] = {x};
  *st = k_mdot<double>(w.rs, src, 0, x, w.n, true, w.dscal, s);
  if (*st) return 0;
  *st = sync_read(w, 1, s);
  return std::sqrt(w.hscal[0]);
}

template <typename T>
static double norm2_t(Workspace& w, const T* x, cudaStream_t s, int* st) {
  const T* src[1] = {x};
  *st = k_mdot<T>(w.rs, src, 0, x, w.n, true, w.dscal, s);
  if (*st) return 0;
  *st = sync_read(w, 1, s);
  return std::sqrt(w.hscal[0]);
}

template <typename T>
static int precond(cheb_plan_s* p, Workspace& w, const LgOpts& lo, const T* r, T* z, cudaStream_t s) {
  if (lo.precond != CHEB_PRECOND_FDM) return k_scale<T>(z, r, 1.0, w.n, s);
  return lo.transpose ? fdm_apply_t<T>(p, w.fdm, lo.kref, r, z, s) : fdm_apply<T>(p, w.fdm, lo.kref, r, z, s);
}

// out = in, with the values at flux-owned boundary nodes divided by -K_p: a
// flux row -K_p s (d_a u)_p = g_p is the Neumann row s (d_a u)_p = -g_p / K_p
__global__ void flux_data_kernel(Geom g, const double* __restrict__ K, const double* __restrict__ in,
                                 double* __restrict__ out) {
  const size_t tot = (size_t)g.n[0] * g.n[1] * g.n[2];
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int k = (int)(c / ((size_t)g.n[0] * g.n[1]));
    const int o = owner_face(g, i, j, k);
    out[c] = (o >= 0 && g.bc[o] == CHEB_FLUX) ? -in[c] / K[c] : in[c];
  }
}

// The paper's formulation (Sec. 2.3.1): the boundary unknowns are eliminated
// (x_r = G x_k + H g per boundary row) and LGMRES runs on the interior
// equations (A_kk + A_kr G) x_k = f_k - A_kr H g, matrix-free: B v =
// P_int A(E_0 v) with E_0 the elimination with zero data, right-hand side
// P_int (b - A E_g(0)), and the solution u = E_g(v).  FP64.
static int solve_eliminated(cheb_plan_s* p, Workspace& w, const double* K, const double* b, double* u,
                            const cheb_solve_opts& o, LgOpts& lo, cheb_solve_info& info, double t0) {
  cudaStream_t s = p->stream;
  const size_t n = w.n;
  int st;
  if ((st = fdm_setup(p, w.fdm))) return st;
  if ((st = ensure_bufs<double>(w, lo.m + lo.k + 1, std::max(1, lo.k)))) return st;
  if (!w.adj[0])
    for (int i = 0; i < 3; ++i) CHEB_CUDA(cudaMalloc(&w.adj[i], sizeof(double) * n));
  if (!w.r64) CHEB_CUDA(cudaMalloc(&w.r64, sizeof(double) * n));
  KrylovBufs<double>& B = w.k64;
  const Geom g = p->geom();
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 8));
  double* rg = w.adj[0];    // boundary data in Neumann form
  double* zero = w.adj[1];  // homogeneous data
  double* v = w.adj[2];     // interior unknowns (full-grid vector)
  flux_data_kernel<<<blocks, 256, 0, s>>>(g, K, b, rg);
  CHEB_LAUNCH_CHECK("flux_data_kernel");
  CHEB_CUDA(cudaMemsetAsync(zero, 0, sizeof(double) * n, s));
  // E_g(0) in B.x, then r64 = P_int (b - A E_g(0))
  CHEB_CUDA(cudaMemsetAsync(B.x, 0, sizeof(double) * n, s));
  if ((st = fdm_fill_boundary<double>(p, w.fdm, rg, B.x, s))) return st;
  if ((st = launch_apply<double>(p, K, B.x, w.r64, s))) return st;
  if ((st = k_residual<double>(w.r64, b, n, s))) return st;
  mask_interior_kernel<<<blocks, 256, 0, s>>>(g, w.r64, w.r64);
  CHEB_LAUNCH_CHECK("mask_interior_kernel");
  lo.elim = true;
  lo.elim_zero = zero;
  // right-hand side c = [M_int^{-1}] P_int (b - A E_g(0))
  if (lo.precond == CHEB_PRECOND_FDM) {
    if ((st = fdm_apply<double>(p, w.fdm, lo.kref, w.r64, B.tmp, s))) return st;
    mask_interior_kernel<<<blocks, 256, 0, s>>>(g, B.tmp, B.c);
  } else {
    mask_interior_kernel<<<blocks, 256, 0, s>>>(g, w.r64, B.c);
  }
  CHEB_LAUNCH_CHECK("mask_interior_kernel");
  const double nb = norm2_dev(w, B.c, s, &st);
  if (st) return st;
  mask_interior_kernel<<<blocks, 256, 0, s>>>(g, u, v);  // initial guess: the interior of u
  CHEB_LAUNCH_CHECK("mask_interior_kernel");
  int rc = CHEB_OK;
  LgStats stt;
  if (nb > 0.0) {
    lo.tol_abs = std::max(o.rtol * nb, o.atol);
    lo.maxiter = o.maxiter;
    rc = lgmres<double>(p, w, lo, K, B.c, v, false, stt, s);
    if (rc < 0) return rc;
  }
  // u = E_g(v)
  CHEB_CUDA(cudaMemcpyAsync(u, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if ((st = fdm_fill_boundary<double>(p, w.fdm, rg, u, s))) return st;
  CHEB_CUDA(cudaStreamSynchronize(s));
  info.iterations = stt.iterations;
  info.cycles = stt.cycles;
  info.applies_fp64 = stt.applies;
  info.host_syncs = stt.syncs;
  info.discarded_steps = stt.overshoot;
  info.rel_residual = nb > 0.0 ? stt.resid / nb : 0.0;
  info.seconds = now_s() - t0;
  info.status = rc;
  return rc;
}

static int solve_impl(cheb_plan_s* p, const double* K, const double* b, double* u,
                      const cheb_solve_opts& o, cheb_solve_info& info, bool transpose = false) {
  const double t0 = now_s();
  cudaStream_t s = p->stream;
  int st;
  bool has_dir = false;
  for (int f = 0; f < 2 * p->dim; ++f) has_dir |= p->bc[f] == CHEB_DIRICHLET;
  if (!has_dir) { set_error("every face is Neumann: the system is singular"); return CHEB_ERR_SINGULAR_BC; }
  if (o.restart < 1 || o.augment < 0 || o.restart + o.augment + 1 > kMaxVecs) {
    set_error("need restart >= 1, augment >= 0, restart + augment < 40"); return CHEB_ERR_ARG;
  }
  if ((st = ensure_ws(p))) return st;
  Workspace& w = *p->ws;
  const size_t n = w.n;
  if (!pmat_ok(o)) return CHEB_ERR_ARG;
  LgOpts lo;
  lo.m = o.restart;
  lo.k = o.augment;
  lo.reorth = o.reorth != 0;
  lo.precond = o.precond;
  lo.pmat = o.precond_matrices;
  lo.transpose = transpose;
  lo.use_graph = o.use_graph != 0;
  if (o.precond == CHEB_PRECOND_FDM) {
    if ((st = fdm_setup(p, w.fdm))) return st;
    if ((st = fdm_clear(w.fdm, s))) return st;
    w.fdm.tf32_mats = o.precond_matrices == CHEB_PMAT_TF32;
    if (o.kref > 0) lo.kref = o.kref;
    else {
      if ((st = k_sum_log(w.rs, K, n, w.dscal, s))) return st;
      if ((st = sync_read(w, 1, s))) return st;
      lo.kref = std::exp(w.hscal[0] / (double)n);
    }
  }
  info.kref = lo.kref;
  if (o.formulation == CHEB_FORM_ELIMINATE) {
    if (o.mode != CHEB_SOLVE_FP64 || transpose) {
      set_error("the elimination formulation is FP64 forward solves only");
      return CHEB_ERR_UNSUPPORTED;
    }
    return solve_eliminated(p, w, K, b, u, o, lo, info, t0);
  }
  // ||M^{-1} b||
  double nb;
  if (o.mode == CHEB_SOLVE_FP64) {
    if ((st = ensure_bufs<double>(w, lo.m + lo.k + 1, std::max(1, lo.k)))) return st;
    KrylovBufs<double>& B = w.k64;
    if ((st = precond<double>(p, w, lo, b, B.c, s))) return st;
    nb = norm2_dev(w, B.c, s, &st);
    if (st) return st;
    if (nb == 0.0) {
      CHEB_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * n, s));
      CHEB_CUDA(cudaStreamSynchronize(s));
      info.status = CHEB_OK;
      return CHEB_OK;
    }
    lo.tol_abs = std::max(o.rtol * nb, o.atol);
    lo.maxiter = o.maxiter;
    LgStats stt;
    int rc = lgmres<double>(p, w, lo, K, B.c, u, false, stt, s);
    info.iterations = stt.iterations;
    info.cycles = stt.cycles;
    info.applies_fp64 = stt.applies;
    info.graph_captures = stt.captures;
    info.host_syncs = stt.syncs;
    info.discarded_steps = stt.overshoot;
    info.rel_residual = stt.resid / nb;
    info.seconds = now_s() - t0;
    info.status = rc;
    return rc;
  }
  // ---- mixed: FP32 inner LGMRES inside FP64 iterative refinement
  if ((st = ensure_bufs<float>(w, lo.m + lo.k + 1, std::max(1, lo.k)))) return st;
  KrylovBufs<float>& B = w.k32;
  if (!w.r64) CHEB_CUDA(cudaMalloc(&w.r64, sizeof(double) * n));
  if ((st = k_cast_scale<float, double>(B.K, K, 1.0, n, s))) return st;
  {
    const double sb = norm2_dev(w, b, s, &st);
    if (st) return st;
    if (sb == 0.0) {
      CHEB_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * n, s));
      CHEB_CUDA(cudaStreamSynchronize(s));
      info.status = CHEB_OK;
      return CHEB_OK;
    }
    if ((st = k_cast_scale<float, double>(B.tmp, b, 1.0 / sb, n, s))) return st;
    if ((st = precond<float>(p, w, lo, B.tmp, B.c, s))) return st;
    nb = sb * norm2_t<float>(w, B.c, s, &st);
    if (st) return st;
  }
  int rc = CHEB_ERR_NOT_CONVERGED;
  double eta = 1.0;
  LgCarry carry;  // augmentation vectors reused by the next refinement's inner solve
  for (int it = 0; it <= o.max_refinements; ++it) {
    // r64 = b - A u (FP64)
    prof_begin(kProfApply64, s);
    if ((st = transpose ? launch_adjoint_apply<double>(p, K, u, w.r64, s)
                        : launch_apply<double>(p, K, u, w.r64, s)))
      return st;
    prof_end(kProfApply64, s);
    info.applies_fp64++;
    prof_begin(kProfOther, s);
    if ((st = k_residual<double>(w.r64, b, n, s))) return st;
    const double sr = norm2_dev(w, w.r64, s, &st);
    prof_end(kProfOther, s);
    if (st) return st;
    if (!std::isfinite(sr)) { set_error("non-finite residual"); return CHEB_ERR_NONFINITE; }
    if (sr == 0.0) { eta = 0.0; rc = CHEB_OK; break; }
    prof_begin(kProfOther, s);
    if ((st = k_cast_scale<float, double>(B.tmp, w.r64, 1.0 / sr, n, s))) return st;
    prof_end(kProfOther, s);
    prof_begin(kProfPrec32, s);
    if ((st = precond<float>(p, w, lo, B.tmp, B.c, s))) return st;
    prof_end(kProfPrec32, s);
    prof_begin(kProfOther, s);
    const double cn = norm2_t<float>(w, B.c, s, &st);
    prof_end(kProfOther, s);
    if (st) return st;
    eta = sr * cn / nb;
    if (o.verbose) fprintf(stderr, "[cheb] refinement %d: eta = %.3e\n", it, eta);
    if (eta <= o.rtol || sr * cn <= o.atol) { rc = CHEB_OK; break; }
    if (it == o.max_refinements || info.iterations >= o.maxiter) break;
    LgOpts li = lo;
    // the inner solve reduces its residual by inner_rtol, but by no more than
    // the outer tolerance still asks for (with a factor 2 margin): the last
    // refinement of a solve usually needs far less than inner_rtol
    li.tol_abs = std::max(o.inner_rtol, 0.5 * o.rtol / eta) * cn;
    li.maxiter = std::min(o.inner_maxiter, o.maxiter - info.iterations);
    LgStats stt;
    int r2 = lgmres<float>(p, w, li, B.K, B.c, B.x, true, stt, s, o.recycle ? &carry : nullptr);
    if (r2 < 0) return r2;
    info.iterations += stt.iterations;
    info.cycles += stt.cycles;
    info.applies_fp32 += stt.applies;
    info.graph_captures += stt.captures;
    info.host_syncs += stt.syncs;
    info.discarded_steps += stt.overshoot;
    info.refinements++;
    info.rel_residual_inner = stt.resid / cn;
    prof_begin(kProfOther, s);
    if ((st = k_axpy64<float>(u, B.x, sr, n, s))) return st;
    prof_end(kProfOther, s);
  }
  CHEB_CUDA(cudaStreamSynchronize(s));
  info.rel_residual = eta;
  info.seconds = now_s() - t0;
  info.status = rc;
  return rc;
}

// dJdK += sum_a (D_a^T P_int lam) * (D_a u): the derivative of -lam^T A(K) u
// with respect to K_p, since K enters A only through the interior rows
// -sum_a D_a diag(K) D_a.
__global__ void mask_interior_kernel(Geom g, const double* __restrict__ x, double* __restrict__ y) {
  const size_t tot = (size_t)g.n[0] * g.n[1] * g.n[2];
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int k = (int)(c / ((size_t)g.n[0] * g.n[1]));
    bool b = (i == 0 || i == g.n[0] - 1);
    if (g.dim > 1) b = b || j == 0 || j == g.n[1] - 1;
    if (g.dim > 2) b = b || k == 0 || k == g.n[2] - 1;
    y[c] = b ? 0.0 : x[c];
  }
}

__global__ void fma_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y,
                           size_t n) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    y[c] += a[c] * b[c];
}

// flux rows -K_p s (D_a u)_p depend on K_p: dJdK_p += s lam_p (D_a u)_p on the
// rows owned by a flux face of axis a
__global__ void flux_grad_kernel(Geom g, int axis, const double* __restrict__ lam, const double* __restrict__ du,
                                 double* __restrict__ dJdK) {
  const size_t tot = (size_t)g.n[0] * g.n[1] * g.n[2];
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int k = (int)(c / ((size_t)g.n[0] * g.n[1]));
    const int o = owner_face(g, i, j, k);
    if (o >= 0 && (o >> 1) == axis && g.bc[o] == CHEB_FLUX)
      dJdK[c] += ((o & 1) ? 1.0 : -1.0) * lam[c] * du[c];
  }
}

static int grad_K_accumulate(cheb_plan_s* p, const double* u, const double* lam, double* dJdK) {
  int st;
  if ((st = ensure_ws(p))) return st;
  Workspace& w = *p->ws;
  const size_t n = w.n;
  if (!w.adj[0])
    for (int i = 0; i < 3; ++i) CHEB_CUDA(cudaMalloc(&w.adj[i], sizeof(double) * n));
  cudaStream_t s = p->stream;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 8));
  mask_interior_kernel<<<blocks, 256, 0, s>>>(p->geom(), lam, w.adj[0]);
  CHEB_LAUNCH_CHECK("mask_interior_kernel");
  for (int a = 0; a < p->dim; ++a) {
    if ((st = launch_pass<double>(p, a, kDerivT, nullptr, w.adj[0], w.adj[1], s))) return st;
    if ((st = launch_pass<double>(p, a, kDeriv, nullptr, u, w.adj[2], s))) return st;
    fma_kernel<<<blocks, 256, 0, s>>>(w.adj[1], w.adj[2], dJdK, n);
    CHEB_LAUNCH_CHECK("fma_kernel");
    if (has_flux(p)) {
      flux_grad_kernel<<<blocks, 256, 0, s>>>(p->geom(), a, lam, w.adj[2], dJdK);
      CHEB_LAUNCH_CHECK("flux_grad_kernel");
    }
  }
  return CHEB_OK;
}

// K = K0 (1 + beta |grad u|^2) from the three gradient components g0, g1, g2
__global__ void picard_k_kernel(const double* __restrict__ K0, const double* __restrict__ g0,
                                const double* __restrict__ g1, const double* __restrict__ g2, int dim,
                                double beta, double* __restrict__ K, size_t n) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    double s = g0[c] * g0[c];
    if (dim > 1) s += g1[c] * g1[c];
    if (dim > 2) s += g2[c] * g2[c];
    K[c] = K0[c] * (1.0 + beta * s);
  }
}

static int picard_conductivity(cheb_plan_s* p, const double* K0, const double* u, double beta, double* K) {
  Workspace& w = *p->ws;
  const size_t n = w.n;
  int st;
  for (int a = 0; a < p->dim; ++a)
    if ((st = launch_pass<double>(p, a, kDeriv, nullptr, u, w.adj[a], p->stream))) return st;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 8));
  picard_k_kernel<<<blocks, 256, 0, p->stream>>>(K0, w.adj[0], w.adj[1], w.adj[2], p->dim, beta, K, n);
  CHEB_LAUNCH_CHECK("picard_k_kernel");
  return CHEB_OK;
}

// Picard iteration (Sec. 2.3, Picard): the nonlinearity is frozen at the
// previous iterate, K^m = K0 (1 + beta |grad u^m|^2), the linear system
// A(K^m) u* = b is solved warm-started from u^m, and u^{m+1} = omega u* +
// (1 - omega) u^m (omega = 1: the plain iteration); stop when
// ||u^{m+1} - u^m|| / ||u^{m+1}|| <= tol or after maxit outer steps.
__global__ void relax_kernel(double* __restrict__ u, const double* __restrict__ uprev, double omega,
                             size_t n) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    u[c] = omega * u[c] + (1.0 - omega) * uprev[c];
}

static int picard_impl(cheb_plan_s* p, const double* K0, const double* b, double* u, double beta,
                       double omega, double tol, int maxit, const cheb_solve_opts& o,
                       cheb_solve_info& info, int* iters, double* delta) {
  int st;
  if ((st = ensure_ws(p))) return st;
  Workspace& w = *p->ws;
  const size_t n = w.n;
  if (!w.adj[0])
    for (int i = 0; i < 3; ++i) CHEB_CUDA(cudaMalloc(&w.adj[i], sizeof(double) * n));
  if (!w.picK) {
    CHEB_CUDA(cudaMalloc(&w.picK, sizeof(double) * n));
    CHEB_CUDA(cudaMalloc(&w.picU, sizeof(double) * n));
  }
  int rc = CHEB_ERR_NOT_CONVERGED;
  double d = 1.0;
  int m = 0;
  cheb_solve_info tot;
  std::memset(&tot, 0, sizeof(tot));
  const double t0 = now_s();
  cheb_solve_opts oi = o;  // kref frozen after the first step: captured graphs stay valid
  for (m = 1; m <= maxit; ++m) {
    if ((st = picard_conductivity(p, K0, u, beta, w.picK))) return st;
    CHEB_CUDA(cudaMemcpyAsync(w.picU, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->stream));
    cheb_solve_info li;
    std::memset(&li, 0, sizeof(li));
    int r = solve_impl(p, w.picK, b, u, oi, li);
    if (oi.kref <= 0) oi.kref = li.kref;
    tot.iterations += li.iterations;
    tot.cycles += li.cycles;
    tot.refinements += li.refinements;
    tot.applies_fp64 += li.applies_fp64;
    tot.applies_fp32 += li.applies_fp32;
    tot.host_syncs += li.host_syncs;
    tot.discarded_steps += li.discarded_steps;
    tot.rel_residual = li.rel_residual;
    tot.kref = li.kref;
    if (r < 0) return r;
    if (omega != 1.0) {
      const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 8));
      relax_kernel<<<blocks, 256, 0, p->stream>>>(u, w.picU, omega, n);
      CHEB_LAUNCH_CHECK("relax_kernel");
    }
    if ((st = cheb_rel_diff(p, u, w.picU, &d))) return st;
    if (o.verbose) fprintf(stderr, "[cheb] picard %d: |du|/|u| = %.3e (%d its)\n", m, d, li.iterations);
    if (d <= tol) { rc = CHEB_OK; break; }
  }
  tot.seconds = now_s() - t0;
  tot.status = rc;
  info = tot;
  if (iters) *iters = std::min(m, maxit);
  if (delta) *delta = d;
  return rc;
}

// Newton coefficients of k(u) = K0 / (1 + alpha u): K = k(u) and, from the
// derivatives d_a u held in C[a], C[a] = k'(u) d_a u = -alpha K / (1 + alpha u) d_a u.
__global__ void newton_coeff_kernel(const double* __restrict__ K0, const double* __restrict__ u, double alpha,
                                    int dim, double* __restrict__ K, double* __restrict__ C0,
                                    double* __restrict__ C1, double* __restrict__ C2, size_t n) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const double d = 1.0 + alpha * u[c];
    const double k = K0[c] / d;
    const double dk = -alpha * k / d;
    K[c] = k;
    C0[c] *= dk;
    if (dim > 1) C1[c] *= dk;
    if (dim > 2) C2[c] *= dk;
  }
}

struct NewtonBufs {
  double* K = nullptr;
  double* C[3] = {nullptr, nullptr, nullptr};
  double* r = nullptr;     // -R(u) = b - A(k(u)) u
  double* du = nullptr;    // FP64 Newton step
  float* K32 = nullptr;
  float* C32[3] = {nullptr, nullptr, nullptr};
};

static int newton_impl(cheb_plan_s* p, const double* K0, double alpha, const double* b, double* u, double tol,
                       int maxit, const cheb_solve_opts& o, cheb_solve_info& info, int* iters, double* delta) {
  const double t0 = now_s();
  cudaStream_t s = p->stream;
  int st;
  bool has_dir = false;
  for (int f = 0; f < 2 * p->dim; ++f) has_dir |= p->bc[f] == CHEB_DIRICHLET;
  if (!has_dir) { set_error("no Dirichlet face: the linearised system is singular"); return CHEB_ERR_SINGULAR_BC; }
  if (o.restart < 1 || o.augment < 0 || o.restart + o.augment + 1 > kMaxVecs) {
    set_error("need restart >= 1, augment >= 0, restart + augment < 40"); return CHEB_ERR_ARG;
  }
  if (!pmat_ok(o)) return CHEB_ERR_ARG;
  if ((st = ensure_ws(p))) return st;
  Workspace& w = *p->ws;
  const size_t n = w.n;
  const bool mixed = o.mode == CHEB_SOLVE_MIXED;
  // scratch: K, C_a, residual and step in FP64; FP32 copies for mixed mode
  NewtonBufs nb;
  auto release = [&]() {
    cudaFree(nb.K); cudaFree(nb.r); cudaFree(nb.du); cudaFree(nb.K32);
    for (int a = 0; a < 3; ++a) { cudaFree(nb.C[a]); cudaFree(nb.C32[a]); }
  };
  struct Guard { std::function<void()> f; ~Guard() { f(); } } guard{release};
  CHEB_CUDA(cudaMalloc(&nb.K, sizeof(double) * n));
  CHEB_CUDA(cudaMalloc(&nb.r, sizeof(double) * n));
  CHEB_CUDA(cudaMalloc(&nb.du, sizeof(double) * n));
  for (int a = 0; a < 3; ++a) CHEB_CUDA(cudaMalloc(&nb.C[a], sizeof(double) * n));
  if (mixed) {
    CHEB_CUDA(cudaMalloc(&nb.K32, sizeof(float) * n));
    for (int a = 0; a < 3; ++a) CHEB_CUDA(cudaMalloc(&nb.C32[a], sizeof(float) * n));
  }
  if (o.precond == CHEB_PRECOND_FDM) {
    if ((st = fdm_setup(p, w.fdm))) return st;
    if ((st = fdm_clear(w.fdm, s))) return st;
    w.fdm.tf32_mats = o.precond_matrices == CHEB_PMAT_TF32;
  }
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 148 * 8));
  int rc = CHEB_ERR_NOT_CONVERGED;
  double d = 1.0;
  int m = 0;
  for (m = 1; m <= maxit; ++m) {
    // K = k(u), C_a = k'(u) d_a u
    for (int a = 0; a < p->dim; ++a)
      if ((st = launch_pass<double>(p, a, kDeriv, nullptr, u, nb.C[a], s))) return st;
    newton_coeff_kernel<<<blocks, 256, 0, s>>>(K0, u, alpha, p->dim, nb.K, nb.C[0], nb.C[1], nb.C[2], n);
    CHEB_LAUNCH_CHECK("newton_coeff_kernel");
    // -R(u) = b - A(K) u (FP64, boundary rows included)
    prof_begin(kProfApply64, s);
    if ((st = launch_apply<double>(p, nb.K, u, nb.r, s))) return st;
    prof_end(kProfApply64, s);
    info.applies_fp64++;
    if ((st = k_residual<double>(nb.r, b, n, s))) return st;
    const double sr = norm2_dev(w, nb.r, s, &st);
    if (st) return st;
    if (!std::isfinite(sr)) { set_error("non-finite Newton residual"); return CHEB_ERR_NONFINITE; }
    if (sr == 0.0) { d = 0.0; rc = CHEB_OK; break; }
    LgOpts lo;
    lo.m = o.restart;
    lo.k = o.augment;
    lo.reorth = o.reorth != 0;
    lo.precond = o.precond;
    lo.pmat = o.precond_matrices;
    if (o.precond == CHEB_PRECOND_FDM) {
      if (o.kref > 0) lo.kref = o.kref;
      else {
        if ((st = k_sum_log(w.rs, nb.K, n, w.dscal, s))) return st;
        if ((st = sync_read(w, 1, s))) return st;
        lo.kref = std::exp(w.hscal[0] / (double)n);
      }
    }
    info.kref = lo.kref;
    // converged already when the preconditioned nonlinear residual meets the
    // solve tolerance: ||M^{-1} R(u)|| <= rtol ||M^{-1} b|| (e.g. a prolonged
    // guess from a coarser level that resolved the solution)
    {
      if ((st = ensure_bufs<double>(w, lo.m + lo.k + 1, std::max(1, lo.k)))) return st;
      KrylovBufs<double>& B = w.k64;
      if ((st = precond<double>(p, w, lo, nb.r, B.c, s))) return st;
      const double rn = norm2_dev(w, B.c, s, &st);
      if (st) return st;
      if ((st = precond<double>(p, w, lo, b, B.tmp, s))) return st;
      const double bn = norm2_dev(w, B.tmp, s, &st);
      if (st) return st;
      info.rel_residual = bn > 0 ? rn / bn : rn;
      if (!std::isfinite(rn)) { set_error("non-finite Newton residual"); return CHEB_ERR_NONFINITE; }
      if (rn <= o.rtol * bn || rn <= o.atol) { d = 0.0; rc = CHEB_OK; break; }
    }
    LgStats stt;
    double step_norm = 0.0;
    if (!mixed) {
      if ((st = ensure_bufs<double>(w, lo.m + lo.k + 1, std::max(1, lo.k)))) return st;
      KrylovBufs<double>& B = w.k64;
      for (int a = 0; a < 3; ++a) lo.jac[a] = nb.C[a < p->dim ? a : 0];
      if ((st = precond<double>(p, w, lo, nb.r, B.c, s))) return st;
      const double cn = norm2_dev(w, B.c, s, &st);
      if (st) return st;
      lo.tol_abs = o.inner_rtol * cn;
      lo.maxiter = std::min(o.inner_maxiter, std::max(1, o.maxiter - info.iterations));
      int r2 = lgmres<double>(p, w, lo, nb.K, B.c, nb.du, true, stt, s);
      if (r2 < 0) return r2;
      step_norm = norm2_dev(w, nb.du, s, &st);
      if (st) return st;
      if ((st = k_axpy64<double>(u, nb.du, 1.0, n, s))) return st;
      info.applies_fp64 += stt.applies;
    } else {
      if ((st = ensure_bufs<float>(w, lo.m + lo.k + 1, std::max(1, lo.k)))) return st;
      KrylovBufs<float>& B = w.k32;
      if ((st = k_cast_scale<float, double>(nb.K32, nb.K, 1.0, n, s))) return st;
      for (int a = 0; a < p->dim; ++a)
        if ((st = k_cast_scale<float, double>(nb.C32[a], nb.C[a], 1.0, n, s))) return st;
      for (int a = 0; a < 3; ++a) lo.jac[a] = nb.C32[a < p->dim ? a : 0];
      if ((st = k_cast_scale<float, double>(B.tmp, nb.r, 1.0 / sr, n, s))) return st;
      if ((st = precond<float>(p, w, lo, B.tmp, B.c, s))) return st;
      const double cn = norm2_t<float>(w, B.c, s, &st);
      if (st) return st;
      lo.tol_abs = o.inner_rtol * cn;
      lo.maxiter = std::min(o.inner_maxiter, std::max(1, o.maxiter - info.iterations));
      int r2 = lgmres<float>(p, w, lo, nb.K32, B.c, B.x, true, stt, s);
      if (r2 < 0) return r2;
      step_norm = sr * norm2_t<float>(w, B.x, s, &st);
      if (st) return st;
      if ((st = k_axpy64<float>(u, B.x, sr, n, s))) return st;
      info.applies_fp32 += stt.applies;
      info.refinements++;
    }
    info.iterations += stt.iterations;
    info.cycles += stt.cycles;
    info.host_syncs += stt.syncs;
    info.discarded_steps += stt.overshoot;
    info.rel_residual_inner = stt.resid;
    const double un = norm2_dev(w, u, s, &st);
    if (st) return st;
    d = un > 0 ? step_norm / un : step_norm;
    if (!std::isfinite(d)) { set_error("non-finite Newton step"); return CHEB_ERR_NONFINITE; }
    if (o.verbose) fprintf(stderr, "[cheb] newton %d: |du|/|u| = %.3e (%d its)\n", m, d, stt.iterations);
    if (d <= tol) { rc = CHEB_OK; break; }
  }
  CHEB_CUDA(cudaStreamSynchronize(s));
  info.seconds = now_s() - t0;
  info.status = rc;
  if (iters) *iters = std::min(m, maxit);
  if (delta) *delta = d;
  return rc;
}

}  // namespace cheb

using namespace cheb;

extern "C" {

static int tensor_core_status(cheb_plan p, int rc);

int cheb_jacobian_apply(cheb_plan p, int prec, const void* K, const void* const C[3], const void* du, void* Jdu) {
  if (!p || !K || !C || !du || !Jdu) { set_error("null argument"); return CHEB_ERR_ARG; }
  for (int a = 0; a < p->dim; ++a)
    if (!C[a]) { set_error("null coefficient field of an active axis"); return CHEB_ERR_ARG; }
  if (Jdu == du || Jdu == K) { set_error("output must not alias K or du"); return CHEB_ERR_ARG; }
  if (prec == CHEB_FP64) {
    const double* c[3] = {(const double*)C[0], (const double*)(p->dim > 1 ? C[1] : C[0]),
                          (const double*)(p->dim > 2 ? C[2] : C[0])};
    return launch_jacobian<double>(p, (const double*)K, c, (const double*)du, (double*)Jdu, p->stream);
  }
  if (prec == CHEB_FP32) {
    const float* c[3] = {(const float*)C[0], (const float*)(p->dim > 1 ? C[1] : C[0]),
                         (const float*)(p->dim > 2 ? C[2] : C[0])};
    return launch_jacobian<float>(p, (const float*)K, c, (const float*)du, (float*)Jdu, p->stream);
  }
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}

int cheb_newton_solve(cheb_plan p, const double* K0, double alpha, const double* b, double* u, double tol,
                      int maxit, const cheb_solve_opts* opts, cheb_solve_info* info, int* newton_iters,
                      double* newton_delta) {
  if (!p || !K0 || !b || !u || maxit < 1 || !(tol > 0) || !std::isfinite(alpha)) {
    set_error("bad argument (need maxit >= 1, tol > 0, finite alpha)");
    return CHEB_ERR_ARG;
  }
  cheb_solve_opts o;
  if (opts) o = *opts;
  else default_opts(o);
  if (o.mode != CHEB_SOLVE_FP64 && o.mode != CHEB_SOLVE_MIXED) { set_error("bad mode"); return CHEB_ERR_ARG; }
  cheb_solve_info tmp;
  std::memset(&tmp, 0, sizeof(tmp));
  int rc = newton_impl(p, K0, alpha, b, u, tol, maxit, o, tmp, newton_iters, newton_delta);
  if (rc >= 0 && (rc = tensor_core_status(p, rc)) < 0) tmp.status = rc;
  if (info) *info = tmp;
  return rc;
}

void cheb_solve_opts_default(cheb_solve_opts* o) {
  if (o) default_opts(*o);
}

// rc, or CHEB_ERR_CUDA when a tensor-core contraction of this plan's
// preconditioner gave up a bounded wait (its output is then invalid).
static int tensor_core_status(cheb_plan p, int rc) {
  if (!p->ws || !p->ws->fdm.rot) return rc;
  const int e = umma_take_error();
  if (e == 0) return rc;
  set_error(e < 0 ? "could not read the tensor-core error word"
                  : "tensor-core contraction: a bounded pipeline wait gave up");
  return CHEB_ERR_CUDA;
}

int cheb_solve(cheb_plan p, const double* K, const double* b, double* u, const cheb_solve_opts* opts,
               cheb_solve_info* info) {
  if (!p || !K || !b || !u) { set_error("null argument"); return CHEB_ERR_ARG; }
  cheb_solve_opts o;
  if (opts) o = *opts;
  else default_opts(o);
  if (o.mode != CHEB_SOLVE_FP64 && o.mode != CHEB_SOLVE_MIXED) { set_error("bad mode"); return CHEB_ERR_ARG; }
  if (o.precond != CHEB_PRECOND_NONE && o.precond != CHEB_PRECOND_FDM) {
    set_error("bad preconditioner"); return CHEB_ERR_ARG;
  }
  cheb_solve_info tmp;
  std::memset(&tmp, 0, sizeof(tmp));
  int rc = solve_impl(p, K, b, u, o, tmp);
  if (rc >= 0 && (rc = tensor_core_status(p, rc)) < 0) tmp.status = rc;
  if (info) *info = tmp;
  return rc;
}

int cheb_prolong(cheb_plan coarse, cheb_plan fine, int prec, const void* uc, void* uf) {
  if (!uc || !uf) { set_error("null argument"); return CHEB_ERR_ARG; }
  int st;
  if ((st = check_prolong_pair(coarse, fine))) return st;
  if ((st = ensure_ws(fine))) return st;
  Workspace& w = *fine->ws;
  if (!w.pro[0]) {
    // intermediates of the axis passes: after x (nx_f, ny_c, nz_c), after y
    // (nx_f, ny_f, nz_c); the larger one sizes both scratch arrays
    const size_t n1 = (size_t)fine->n[0] * coarse->n[1] * coarse->n[2];
    const size_t n2 = (size_t)fine->n[0] * fine->n[1] * coarse->n[2];
    const size_t cap = std::max<size_t>(1, std::max(n1, n2));
    CHEB_CUDA(cudaMalloc(&w.pro[0], sizeof(double) * cap));
    CHEB_CUDA(cudaMalloc(&w.pro[1], sizeof(double) * cap));
  }
  if (prec == CHEB_FP64) {
    prof_begin(kProfProlong, fine->stream);
    st = launch_prolong<double>(coarse, fine, (const double*)uc, (double*)uf, w.pro[0], w.pro[1],
                                fine->stream);
    prof_end(kProfProlong, fine->stream);
    return st;
  }
  if (prec == CHEB_FP32)
    return launch_prolong<float>(coarse, fine, (const float*)uc, (float*)uf, (float*)w.pro[0],
                                 (float*)w.pro[1], fine->stream);
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}

int cheb_rel_diff(cheb_plan p, const double* a, const double* b, double* out) {
  if (!p || !a || !b || !out) { set_error("null argument"); return CHEB_ERR_ARG; }
  int st;
  if ((st = ensure_ws(p))) return st;
  Workspace& w = *p->ws;
  // |a - b|^2 from |a|^2, <a, b>, |b|^2 loses digits: form the difference vector
  if (!w.r64) CHEB_CUDA(cudaMalloc(&w.r64, sizeof(double) * w.n));
  const double* one[1] = {a};
  double cf[2] = {1.0, -1.0};
  const double* two[2] = {a, b};
  if ((st = k_maxpy<double>(w.rs, two, cf, 2, 0.0, w.r64, w.n, w.dscal + 1, p->stream))) return st;
  if ((st = k_mdot<double>(w.rs, one, 0, a, w.n, true, w.dscal, p->stream))) return st;
  if ((st = sync_read(w, 2, p->stream))) return st;
  *out = w.hscal[0] > 0 ? std::sqrt(w.hscal[1] / w.hscal[0]) : 0.0;
  return CHEB_OK;
}

int cheb_solve_hierarchy(int levels, const cheb_plan* plans, const double* const* K,
                         const double* const* b, double* const* u, const cheb_solve_opts* opts,
                         cheb_solve_info* infos, double* e_ref) {
  if (levels < 1 || !plans || !K || !b || !u) { set_error("bad argument"); return CHEB_ERR_ARG; }
  int rc = CHEB_OK, st;
  for (int l = 0; l < levels; ++l) {
    cheb_plan p = plans[l];
    if (l > 0) {
      if ((st = cheb_prolong(plans[l - 1], p, CHEB_FP64, u[l - 1], u[l]))) return st;
      Workspace& w = *p->ws;
      if (!w.pro[2]) CHEB_CUDA(cudaMalloc(&w.pro[2], sizeof(double) * w.n));
      CHEB_CUDA(cudaMemcpyAsync(w.pro[2], u[l], sizeof(double) * w.n, cudaMemcpyDeviceToDevice, p->stream));
    }
    cheb_solve_info info;
    cheb_solve_opts ol;
    if (opts) ol = *opts;
    else default_opts(ol);
    if (l + 1 < levels && ol.coarse_rtol > 0) ol.rtol = ol.coarse_rtol;
    rc = cheb_solve(p, K[l], b[l], u[l], &ol, &info);
    if (infos) infos[l] = info;
    if (rc < 0) return rc;
    if (e_ref) {
      e_ref[l] = 0.0;
      if (l > 0 && (st = cheb_rel_diff(p, u[l], p->ws->pro[2], &e_ref[l]))) return st;
    }
  }
  return rc;
}

}  // extern "C"

// coarse[k][j][i] = fine[r k][r j][r i] (restriction by injection: CGL nodes
// nest, coarse node j is fine node r j for N_fine = r N_coarse)
__global__ void inject_kernel(const double* __restrict__ fine, int fnx, int fny, int r, int cnx, int cny, int cnz,
                              int dim, double* __restrict__ coarse) {
  const size_t tot = (size_t)cnx * cny * cnz;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % cnx);
    const int j = (int)((c / cnx) % cny);
    const int k = (int)(c / ((size_t)cnx * cny));
    const size_t fi = (size_t)i * r;
    const size_t fj = dim > 1 ? (size_t)j * r : 0;
    const size_t fk = dim > 2 ? (size_t)k * r : 0;
    coarse[c] = fine[(fk * fny + fj) * fnx + fi];
  }
}

extern "C" {

int cheb_solve_hierarchy_fine(int levels, const cheb_plan* plans, const double* K, const double* b, double* u,
                              const cheb_solve_opts* opts, cheb_solve_info* infos, double* e_ref) {
  if (levels < 1 || !plans || !K || !b || !u) { set_error("bad argument"); return CHEB_ERR_ARG; }
  cheb_plan pf = plans[levels - 1];
  for (int l = 0; l + 1 < levels; ++l) {
    int st = check_prolong_pair(plans[l], plans[l + 1]);
    if (st) return st;
  }
  int st;
  std::vector<const double*> Kl(levels), bl(levels);
  std::vector<double*> ul(levels);
  for (int l = 0; l < levels; ++l) {
    cheb_plan p = plans[l];
    if (l == levels - 1) { Kl[l] = K; bl[l] = b; ul[l] = u; continue; }
    if ((st = ensure_ws(p))) return st;
    Workspace& w = *p->ws;
    for (int i = 0; i < 3; ++i)
      if (!w.lvl[i]) CHEB_CUDA(cudaMalloc(&w.lvl[i], sizeof(double) * w.n));
    const int r = (pf->n[0] - 1) / (p->n[0] - 1);
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>((w.n + 255) / 256, 148 * 8));
    inject_kernel<<<blocks, 256, 0, pf->stream>>>(K, pf->n[0], pf->n[1], r, p->n[0], p->n[1], p->n[2], p->dim,
                                                  w.lvl[0]);
    CHEB_LAUNCH_CHECK("inject_kernel");
    inject_kernel<<<blocks, 256, 0, pf->stream>>>(b, pf->n[0], pf->n[1], r, p->n[0], p->n[1], p->n[2], p->dim,
                                                  w.lvl[1]);
    CHEB_LAUNCH_CHECK("inject_kernel");
    Kl[l] = w.lvl[0];
    bl[l] = w.lvl[1];
    ul[l] = w.lvl[2];
  }
  // the coarsest level starts from zero; every plan orders its work after the injections
  CHEB_CUDA(cudaMemsetAsync(ul[0], 0, sizeof(double) * plans[0]->size(), pf->stream));
  CHEB_CUDA(cudaStreamSynchronize(pf->stream));
  return cheb_solve_hierarchy(levels, plans, Kl.data(), bl.data(), ul.data(), opts, infos, e_ref);
}

int cheb_precond_apply_t(cheb_plan p, int prec, double kref, const void* y, void* z) {
  if (!p || !y || !z || !(kref > 0)) { set_error("bad argument"); return CHEB_ERR_ARG; }
  int st;
  if ((st = ensure_ws(p))) return st;
  if ((st = fdm_setup(p, p->ws->fdm))) return st;
  if ((st = fdm_clear(p->ws->fdm, p->stream))) return st;
  p->ws->fdm.tf32_mats = false;  // FP32: the matrices to FP32 accuracy
  if (prec == CHEB_FP64) return fdm_apply_t<double>(p, p->ws->fdm, kref, (const double*)y, (double*)z, p->stream);
  if (prec == CHEB_FP32) {
    st = fdm_apply_t<float>(p, p->ws->fdm, kref, (const float*)y, (float*)z, p->stream);
    if (st) return st;
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    return tensor_core_status(p, CHEB_OK);
  }
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}

int cheb_adjoint_solve(cheb_plan p, const double* K, const double* u, const double* dJdu,
                       const cheb_solve_opts* opts, double* lambda, double* dJdK,
                       cheb_solve_info* info) {
  if (!p || !K || !dJdu || !lambda) { set_error("null argument"); return CHEB_ERR_ARG; }
  if (dJdK && !u) { set_error("dJdK needs the forward solution u"); return CHEB_ERR_ARG; }
  cheb_solve_opts o;
  if (opts) o = *opts;
  else default_opts(o);
  cheb_solve_info tmp;
  std::memset(&tmp, 0, sizeof(tmp));
  int rc = solve_impl(p, K, dJdu, lambda, o, tmp, true);
  if (info) *info = tmp;
  if (rc < 0 || !dJdK) return rc;
  int st;
  if ((st = grad_K_accumulate(p, u, lambda, dJdK))) return st;
  return rc;
}

int cheb_picard_solve(cheb_plan p, const double* K0, const double* b, double* u, double beta,
                      double omega, double tol, int maxit, const cheb_solve_opts* opts,
                      cheb_solve_info* info, int* picard_iters, double* picard_delta) {
  if (!p || !K0 || !b || !u || maxit < 1 || !(tol > 0) || !(omega > 0 && omega <= 1)) {
    set_error("bad argument (need maxit >= 1, tol > 0, 0 < omega <= 1)");
    return CHEB_ERR_ARG;
  }
  cheb_solve_opts o;
  if (opts) o = *opts;
  else default_opts(o);
  cheb_solve_info tmp;
  std::memset(&tmp, 0, sizeof(tmp));
  int rc = picard_impl(p, K0, b, u, beta, omega, tol, maxit, o, tmp, picard_iters, picard_delta);
  if (info) *info = tmp;
  return rc;
}

// Independent instances solved concurrently: one host thread per instance,
// each ordering its work on its plan's stream (a private non-blocking
// stream is created for plans on the legacy stream).  K0 and beta select the
// Picard form (K0 != NULL), otherwise K is the fixed conductivity.
static int batched(int count, const cheb_plan* plans, const double* const* K, const double* const* b,
                   double* const* u, const cheb_solve_opts* opts, cheb_solve_info* infos, double beta,
                   double omega, double tol, int maxit, int* iters, bool picard) {
  if (count < 1 || !plans || !K || !b || !u) { set_error("bad argument"); return CHEB_ERR_ARG; }
  int dev = 0;
  CHEB_CUDA(cudaGetDevice(&dev));
  std::vector<int> rcs(count, CHEB_OK);
  std::vector<std::string> errs(count);
  std::vector<std::thread> th;
  for (int i = 0; i < count; ++i) {
    th.emplace_back([&, i]() {
      cudaSetDevice(dev);
      cheb_plan p = plans[i];
      cudaStream_t own = nullptr, saved = p->stream;
      if (!saved) {
        cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking);
        p->stream = own;
      }
      cheb_solve_info inf;
      std::memset(&inf, 0, sizeof(inf));
      int rc;
      if (picard)
        rc = cheb_picard_solve(p, K[i], b[i], u[i], beta, omega, tol, maxit, opts, &inf,
                               iters ? &iters[i] : nullptr, nullptr);
      else
        rc = cheb_solve(p, K[i], b[i], u[i], opts, &inf);
      if (rc < 0) errs[i] = cheb_last_error();
      if (own) {
        cudaStreamSynchronize(own);
        p->stream = saved;
        cudaStreamDestroy(own);
      }
      rcs[i] = rc;
      if (infos) infos[i] = inf;
    });
  }
  for (auto& t : th) t.join();
  int worst = CHEB_OK;
  for (int i = 0; i < count; ++i) {
    if (rcs[i] < 0 && (worst >= 0 || rcs[i] < worst)) { worst = rcs[i]; set_error(errs[i]); }
    else if (worst == CHEB_OK && rcs[i] > 0) worst = rcs[i];
  }
  return worst;
}

// LOCKSTEP / CONCURRENT choice of a batch (CHEB_ERR_UNSUPPORTED when
// LOCKSTEP is forced on a batch it does not cover)
static int batch_route(int count, const cheb_plan* plans, const cheb_solve_opts& o, bool* lock) {
  if (o.batch_mode != CHEB_BATCH_AUTO && o.batch_mode != CHEB_BATCH_LOCKSTEP &&
      o.batch_mode != CHEB_BATCH_CONCURRENT) {
    set_error("bad batch_mode");
    return CHEB_ERR_ARG;
  }
  if (o.mode != CHEB_SOLVE_FP64 && o.mode != CHEB_SOLVE_MIXED) { set_error("bad mode"); return CHEB_ERR_ARG; }
  bool ok = lockstep_ok(count, plans, o);
  if (o.batch_mode == CHEB_BATCH_LOCKSTEP && !ok) {
    set_error("lockstep batch needs n <= 129, a Dirichlet face, one dimension and device, REPLACE, reorth 0");
    return CHEB_ERR_UNSUPPORTED;
  }
  if (o.batch_mode == CHEB_BATCH_AUTO && ok) {
    // Measured on B300 (Picard batches, 8 steps): lockstep wins where the
    // instances are many or small (64 x 33^3: 3.7x, 32 x 49^3: 1.7x), ties
    // at 16 x 65^3 and trails by 14 % on 16 instances of 33^3 .. 97^3 (mean
    // 363k points), where one solver per instance already fills the GPU.
    size_t tot = 0;
    for (int i = 0; i < count; ++i) tot += plans[i]->size();
    ok = count >= 32 || tot / (size_t)count <= 200000;
  }
  *lock = ok && o.batch_mode != CHEB_BATCH_CONCURRENT;
  return CHEB_OK;
}

int cheb_solve_batched(int count, const cheb_plan* plans, const double* const* K, const double* const* b,
                       double* const* u, const cheb_solve_opts* opts, cheb_solve_info* infos) {
  if (count < 1 || !plans || !K || !b || !u) { set_error("bad argument"); return CHEB_ERR_ARG; }
  cheb_solve_opts o;
  resolve_opts(opts, &o);
  bool lock = false;
  int st;
  if ((st = batch_route(count, plans, o, &lock))) return st;
  if (lock) return lockstep_solve(count, plans, K, b, u, o, infos, false, 0.0, 1.0, 1.0, 1, nullptr);
  return batched(count, plans, K, b, u, &o, infos, 0.0, 1.0, 1.0, 1, nullptr, false);
}

int cheb_picard_batched(int count, const cheb_plan* plans, const double* const* K0,
                        const double* const* b, double* const* u, double beta, double omega,
                        double tol, int maxit, const cheb_solve_opts* opts, cheb_solve_info* infos,
                        int* picard_iters) {
  if (count < 1 || !plans || !K0 || !b || !u) { set_error("bad argument"); return CHEB_ERR_ARG; }
  cheb_solve_opts o;
  resolve_opts(opts, &o);
  bool lock = false;
  int st;
  if ((st = batch_route(count, plans, o, &lock))) return st;
  if (lock) return lockstep_solve(count, plans, K0, b, u, o, infos, true, beta, omega, tol, maxit, picard_iters);
  return batched(count, plans, K0, b, u, &o, infos, beta, omega, tol, maxit, picard_iters, true);
}

int cheb_selftest_bounded_wait(long long wait_cycles) {
  int st = umma_wait_selftest(wait_cycles, nullptr);
  if (st) return st;
  const int e = umma_take_error();
  if (e == 0) { set_error("bounded-wait self-test: the wait did not give up"); return CHEB_OK; }
  set_error(e < 0 ? "could not read the tensor-core error word"
                  : "tensor-core contraction: a bounded pipeline wait gave up (self-test)");
  return CHEB_ERR_CUDA;
}

int cheb_flux_average(cheb_plan p, int axis, const double* K, const double* u, double* out) {
  if (!p || !K || !u || !out || axis < 0 || axis >= p->dim) { set_error("bad argument"); return CHEB_ERR_ARG; }
  int st;
  if ((st = ensure_ws(p))) return st;
  Workspace& w = *p->ws;
  if (!w.adj[0])
    for (int i = 0; i < 3; ++i) CHEB_CUDA(cudaMalloc(&w.adj[i], sizeof(double) * w.n));
  cudaStream_t s = p->stream;
  if ((st = launch_pass<double>(p, axis, kDeriv, nullptr, u, w.adj[0], s))) return st;
  if ((st = k_wsum3(w.rs, K, w.adj[0], p->ax[0].cc64, p->dim > 1 ? p->ax[1].cc64 : nullptr,
                    p->dim > 2 ? p->ax[2].cc64 : nullptr, p->n[0], p->n[1], w.n, w.dscal, s)))
    return st;
  if ((st = sync_read(w, 1, s))) return st;
  double vol = 1.0;
  for (int a = 0; a < p->dim; ++a) vol *= p->hi[a] - p->lo[a];
  *out = w.hscal[0] / vol;
  return CHEB_OK;
}

int cheb_precond_apply(cheb_plan p, int prec, double kref, const void* r, void* z) {
  return cheb_precond_apply_m(p, prec, CHEB_PMAT_FP32, kref, r, z);
}

int cheb_precond_apply_m(cheb_plan p, int prec, int matrices, double kref, const void* r, void* z) {
  if (!p || !r || !z || !(kref > 0)) { set_error("bad argument"); return CHEB_ERR_ARG; }
  if (matrices != CHEB_PMAT_TF32 && matrices != CHEB_PMAT_FP32) {
    set_error("matrices must be CHEB_PMAT_TF32 or CHEB_PMAT_FP32");
    return CHEB_ERR_ARG;
  }
  int st;
  if ((st = ensure_ws(p))) return st;
  if ((st = fdm_setup(p, p->ws->fdm))) return st;
  if ((st = fdm_clear(p->ws->fdm, p->stream))) return st;
  p->ws->fdm.tf32_mats = matrices == CHEB_PMAT_TF32;
  if (prec == CHEB_FP64) return fdm_apply<double>(p, p->ws->fdm, kref, (const double*)r, (double*)z, p->stream);
  if (prec == CHEB_FP32) {
    st = fdm_apply<float>(p, p->ws->fdm, kref, (const float*)r, (float*)z, p->stream);
    if (st) return st;
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    return tensor_core_status(p, CHEB_OK);
  }
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}

}  // extern "C"
