// Internal host-side definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/cheb.h"

namespace cheb {

constexpr int kTileL = 16;      // lines per CTA in the line passes
constexpr int kThreads = 256;   // threads per CTA in the line passes
constexpr int kDenseMaxN = 129; // largest axis size of the dense route
constexpr int kTransformMaxN = 256;

// Per-axis device tables.  The transform route needs the FFT twiddles
// exp(-2 pi i t / P), t < P = 2N; the dense route the differentiation matrix.
struct AxisTables {
  int n = 1;           // points
  int N = 0;           // n - 1
  int P = 0;           // warp FFT length of the transform route: 2N, or for the chirp
                       // form the power of two >= 4N - 1 (at least 8)
  double scale = 1.0;  // 2 / (hi - lo)
  int route = CHEB_ROUTE_TRANSFORM;    // FP64 passes
  int route32 = CHEB_ROUTE_TRANSFORM;  // FP32 passes
  int tile = 16;                       // lines per CTA of the FP64 line passes (8 or 16)
  int tile32 = 16;                     // same for the FP32 line passes
  bool transform_ok = false;
  bool dense_ok = false;
  bool chirp = false;  // transform route by Bluestein's convolution (N not a power of two, or N < 4)
  double2* tw64 = nullptr;  // stage twiddles of the length-P warp FFT
  float2* tw32 = nullptr;
  double2* chirp64 = nullptr;  // chirp route: c_j = exp(-i pi j^2 / 2N), j < 2N
  float2* chirp32 = nullptr;
  double2* bhat64 = nullptr;   // chirp route: FFT_P of the wrapped conj(c) kernel, / P
  float2* bhat32 = nullptr;
  double* D64 = nullptr;   // row-major D (n x n)
  float* D32 = nullptr;
  double* cc64 = nullptr;  // Clenshaw-Curtis weights of the axis (n, physical length)
};

// Line route of an axis when the requested one does not apply (tensor route
// for pass kinds it does not cover): the power-of-two transform, else dense
// where the size allows it, else the chirp transform.
inline int line_route(const AxisTables& t) {
  if (t.transform_ok && !t.chirp) return CHEB_ROUTE_TRANSFORM;
  return t.dense_ok ? CHEB_ROUTE_DENSE : CHEB_ROUTE_TRANSFORM;
}

// Geometry passed by value to kernels.
struct Geom {
  int n[3];
  int dim;
  int bc[6];
};

struct Workspace;    // Krylov / solver workspace (solve.cu)
struct TensorApply;  // tensor-core route resources (umma.cu)

}  // namespace cheb

struct cheb_plan_s {
  int dim = 0;
  int n[3] = {1, 1, 1};
  double lo[3] = {-1, -1, -1};
  double hi[3] = {1, 1, 1};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  cudaStream_t stream = nullptr;
  int device = 0;
  cheb::AxisTables ax[3];
  cheb::Workspace* ws = nullptr;
  cheb::TensorApply* tap = nullptr;
  size_t size() const { return (size_t)n[0] * n[1] * n[2]; }
  cheb::Geom geom() const {
    cheb::Geom g;
    for (int a = 0; a < 3; ++a) g.n[a] = n[a];
    g.dim = dim;
    for (int f = 0; f < 6; ++f) g.bc[f] = bc[f];
    return g;
  }
};

namespace cheb {

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Raise the dynamic shared-memory limit of kernel `func` to at least `bytes`
// on the current device.  The largest value set is remembered per (kernel,
// device), so each device gets its own cudaFuncSetAttribute call.
int ensure_smem_attr(const void* func, size_t bytes);

#define CHEB_CUDA(call)                                   \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return ::cheb::cuda_fail(_e, #call); \
  } while (0)

void count_launch();
void add_launches(long long k);
long long thread_launches();  // launches issued by the calling thread

#define CHEB_LAUNCH_CHECK(what)                           \
  do {                                                    \
    ::cheb::count_launch();                               \
    cudaError_t _e = cudaGetLastError();                  \
    if (_e != cudaSuccess) return ::cheb::cuda_fail(_e, what); \
  } while (0)

// Per-phase device timing with CUDA events (off unless cheb_profile_enable).
enum ProfCat {
  kProfApply64 = 0, kProfApply32, kProfPrec64, kProfPrec32, kProfOrth64, kProfOrth32,
  kProfProlong, kProfOther, kProfNCat
};
void prof_begin(int cat, cudaStream_t s);
void prof_end(int cat, cudaStream_t s);

// Line-pass kinds (apply.cu).
enum PassKind {
  kApplyFirst = 0,  // A u, first axis: writes every node
  kApplyAcc = 1,    // A u, later axes: accumulates interior, writes own Neumann rows
  kDeriv = 2,       // du = D_a u
  kDerivT = 3,      // du = D_a^T u
  kAdjFirst = 4,    // A^T lam, first axis
  kAdjAcc = 5,      // A^T lam, later axes
  kJacFirst = 6,    // Newton Jacobian action J du, first axis (apply with K D_a du + c_a du)
  kJacAcc = 7,      // J du, later axes
};

// true when any active face carries flux data (-K n . grad u = g)
inline bool has_flux(const cheb_plan_s* p);

template <typename T>
int launch_pass(const cheb_plan_s* p, int axis, int kind, const T* K, const T* u, T* out,
                cudaStream_t s, const T* C = nullptr);

inline bool has_flux(const cheb_plan_s* p) {
  for (int f = 0; f < 2 * p->dim; ++f)
    if (p->bc[f] == CHEB_FLUX) return true;
  return false;
}

// Krylov helpers (krylov.cu)
template <typename T>
int launch_apply(const cheb_plan_s* p, const T* K, const T* u, T* out, cudaStream_t s);
template <typename T>
int launch_adjoint_apply(const cheb_plan_s* p, const T* K, const T* lam, T* out, cudaStream_t s);
// J du = A(K) du - sum_a D_a (C_a du) on interior rows, flux rows
// -s (K D_a du + C_a du) (the linearisation of Sec. 3.4); C[a] per axis.
template <typename T>
int launch_jacobian(const cheb_plan_s* p, const T* K, const T* const C[3], const T* du, T* out, cudaStream_t s);

}  // namespace cheb
