// Fast-diagonalization preconditioner (fdm.cu).
#pragma once

#include <vector>

#include "internal.h"

namespace cheb {

struct FdmAxisHost {
  int n = 0, m = 0;                  // points, interior points (n - 2)
  std::vector<double> S, Sinv, lam;  // reduced 1-D operator = S diag(lam) S^{-1}
  std::vector<double> G, Binv, Lh;   // end elimination: u_b = G u_int + Binv g; lifting D2_IB Binv
  std::vector<double> Drow;          // rows 0 and N of D (2 x n)
};

template <typename T>
struct FdmAxisDev {
  T *S = nullptr, *Sinv = nullptr, *ST = nullptr, *SinvT = nullptr, *lam = nullptr;
  T *G = nullptr, *Binv = nullptr, *Lh = nullptr, *Drow = nullptr;
};

struct Fdm {
  bool ready = false;
  int m[3] = {1, 1, 1};   // interior points per axis
  int mp[3] = {1, 1, 1};  // padded to a multiple of 4 (compact-array extents; pad is zero)
  FdmAxisHost host[3];
  FdmAxisDev<double> d64[3];
  FdmAxisDev<float> d32[3];
  double* U64[2] = {nullptr, nullptr};  // compact interior work buffers
  float* U32[2] = {nullptr, nullptr};
  double* Y64 = nullptr;                // transposed application: work copy of the input
  float* Y32 = nullptr;
  // FP32 contractions on the tcgen05 kernel (each contraction along the
  // contiguous axis, output transposed: the axes rotate and three
  // contractions restore the layout).  Per axis, split-TF32 pairs
  // (hi, lo) of S, S^{-1}, S^T, S^{-T}, each umma_n_tile(mp) x mp.
  bool rot = false;
  float* uw[3][8] = {};
  // the contractions use the TF32-rounded matrices alone (hi of each pair:
  // two products per step) instead of the split pairs (three products); set
  // by each solve from its options
  bool tf32_mats = false;
  // batched solves: the kernels of this preconditioner return at entry while
  // *active == 0 (the instance has converged); null outside batches.  The
  // small-grid GEMM contractions (no tcgen05 route) are not masked.
  const int* active = nullptr;
};

int fdm_setup(const cheb_plan_s* p, Fdm& f);
void fdm_free(Fdm& f);
// Re-zero the compact work arrays (both precisions, where allocated).  Their
// zero padding is what the contractions read past the interior; a non-finite
// input leaves 0 * inf = NaN there, so every solve and every direct
// preconditioner call starts from cleared arrays.
int fdm_clear(const Fdm& f, cudaStream_t s);
// x = M^{-1} r with M the constant-kref collocation operator (same boundary rows).
template <typename T>
int fdm_apply(const cheb_plan_s* p, Fdm& f, double kref, const T* r, T* x, cudaStream_t s);
// Boundary values of x from its interior and the boundary data r by the
// per-line elimination of the boundary rows (Sec. 2.3.1: x_r = G x_k + H g):
// faces from their lines' interiors, then edges and corners.  Neumann-type
// rows take r as n.grad x data (flux data must be divided by -K first).
template <typename T>
int fdm_fill_boundary(const cheb_plan_s* p, Fdm& f, const T* r, T* x, cudaStream_t s);
// The allocations fdm_apply<T> makes on first use, made now (a captured
// graph may not allocate).
template <typename T>
int fdm_prepare(const cheb_plan_s* p, Fdm& f, cudaStream_t s);
// Batched steps of lockstep batch solves (FP32, instances with the tcgen05
// route and no flux faces): z = M^{-1} r for every instance of a batch is
// fdm_batch_lift (all instances, one launch), fdm_rot_core per instance,
// fdm_batch_faces (all instances: one launch for the face steps, one per
// boundary-line stage).  Vectors are the batch's concatenated fields
// (instance i at element off[i]); each instance's mask (Fdm::active) is
// read by all of its kernels.
struct FdmBatch;
bool fdm_batchable(const cheb_plan_s* p, const Fdm& f);
int fdm_batch_create(FdmBatch** out, const std::vector<const cheb_plan_s*>& plans, const std::vector<Fdm*>& fdms,
                     const std::vector<long long>& off);
int fdm_batch_kref(FdmBatch* b, const std::vector<double>& kref);
void fdm_batch_free(FdmBatch* b);
int fdm_batch_lift(const FdmBatch* b, const float* rb, cudaStream_t s);
int fdm_batch_faces(const FdmBatch* b, const float* rb, float* xb, cudaStream_t s);
int fdm_rot_core(const cheb_plan_s* p, Fdm& f, double kref, const float* r, float* x, cudaStream_t s);
// z = M^{-T} y (for the adjoint solve).
template <typename T>
int fdm_apply_t(const cheb_plan_s* p, Fdm& f, double kref, const T* y, T* z, cudaStream_t s);

}  // namespace cheb
