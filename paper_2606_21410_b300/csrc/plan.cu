// Plan creation and the plain entry points: nodes, routes, derivative line
// passes, operator apply (forward and transposed), right-hand side.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "hostmath.h"
#include "internal.h"
#include "umma.h"

namespace cheb {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? CHEB_ERR_NOMEM : CHEB_ERR_CUDA;
}

namespace {
std::mutex g_attr_mu;
std::map<std::pair<const void*, int>, size_t> g_attr;  // (kernel, device) -> bytes set
}  // namespace

int ensure_smem_attr(const void* func, size_t bytes) {
  int dev = 0;
  CHEB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_attr_mu);
  size_t& have = g_attr[std::make_pair(func, dev)];
  if (bytes <= have) return CHEB_OK;
  CHEB_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
  return CHEB_OK;
}

int launch_rhs(const cheb_plan_s* p, const double* f, const double* const face_vals[6], double* b,
               cudaStream_t s);
void free_workspace(cheb_plan_s* p);

// ---------------------------------------------------------------------------
// launch counter and phase profiler
// ---------------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void add_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long thread_launches() { return t_launches; }

namespace {
struct ProfRec { int cat; cudaEvent_t a, b; };
struct ProfState {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<ProfRec> recs;
  cudaEvent_t open[kProfNCat] = {};
  double ms[kProfNCat] = {};
  long long cnt[kProfNCat] = {};
};
ProfState g_prof;
std::mutex g_prof_mu;
cudaEvent_t take_event() {
  if (!g_prof.pool.empty()) { cudaEvent_t e = g_prof.pool.back(); g_prof.pool.pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
void collect_locked() {
  for (auto& r : g_prof.recs) {
    cudaEventSynchronize(r.b);
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    g_prof.ms[r.cat] += t;
    g_prof.cnt[r.cat] += 1;
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.recs.clear();
}
}  // namespace

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

void prof_begin(int cat, cudaStream_t s) {
  if (!g_prof.on || capturing(s)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e = take_event();
  cudaEventRecord(e, s);
  g_prof.open[cat] = e;
}

void prof_end(int cat, cudaStream_t s) {
  if (!g_prof.on || capturing(s)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof.open[cat]) return;
  cudaEvent_t e = take_event();
  cudaEventRecord(e, s);
  g_prof.recs.push_back({cat, g_prof.open[cat], e});
  g_prof.open[cat] = nullptr;
  if (g_prof.recs.size() > 4096) collect_locked();
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// In-place forward DFT of length L (a power of two), long double, on the
// host: iterative radix-2 (bit reversal, then butterflies with exact-index
// roots exp(-2 pi i q / L)).
static void host_fft(std::vector<long double>& re, std::vector<long double>& im) {
  const int L = (int)re.size();
  for (int i = 1, j = 0; i < L; ++i) {
    int bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      std::swap(re[i], re[j]);
      std::swap(im[i], im[j]);
    }
  }
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> wr(L / 2), wi(L / 2);
  for (int q = 0; q < L / 2; ++q) {
    wr[q] = cosl(-2.0L * pi * (long double)q / (long double)L);
    wi[q] = sinl(-2.0L * pi * (long double)q / (long double)L);
  }
  for (int len = 2; len <= L; len <<= 1) {
    const int half = len >> 1, step = L / len;
    for (int b = 0; b < L; b += len)
      for (int k = 0; k < half; ++k) {
        const long double cr = wr[k * step], ci = wi[k * step];
        const long double xr = re[b + k + half] * cr - im[b + k + half] * ci;
        const long double xi = re[b + k + half] * ci + im[b + k + half] * cr;
        re[b + k + half] = re[b + k] - xr;
        im[b + k + half] = im[b + k] - xi;
        re[b + k] += xr;
        im[b + k] += xi;
      }
  }
}

// Tables of the chirp-form DFT of length M = 2N with convolution length L
// (Bluestein): c_j = exp(-i pi j^2 / M), j < M, with j^2 reduced mod 2M
// before the angle is formed; bhat = FFT_L(b) / L, b_m = conj(c_m) at
// m and L - m for 0 <= m < M, zero elsewhere.  Long double throughout.
static void chirp_tables(int N, int L, std::vector<double2>& c, std::vector<double2>& bhat) {
  const int M = 2 * N;
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> cr(M), ci(M);
  for (int j = 0; j < M; ++j) {
    const long long r = ((long long)j * j) % (2LL * M);
    const long double ang = -pi * (long double)r / (long double)M;
    cr[j] = cosl(ang);
    ci[j] = sinl(ang);
  }
  c.resize(M);
  for (int j = 0; j < M; ++j) c[j] = make_double2((double)cr[j], (double)ci[j]);
  std::vector<long double> br(L, 0.0L), bi(L, 0.0L);
  for (int m = 0; m < M; ++m) {
    br[m] = cr[m];
    bi[m] = -ci[m];  // conj(c_m)
    if (m > 0) {
      br[L - m] = cr[m];
      bi[L - m] = -ci[m];
    }
  }
  host_fft(br, bi);
  bhat.resize(L);
  for (int k = 0; k < L; ++k) bhat[k] = make_double2((double)(br[k] / L), (double)(bi[k] / L));
}

// Reference CGL coordinate x_j = cos(pi j / N), evaluated as
// sin(pi (N - 2j) / (2N)) (same value; exactly antisymmetric).
static double cgl_ref(int j, int N) { return std::sin(M_PI * (double)(N - 2 * j) / (2.0 * N)); }

static int build_axis(cheb_plan_s* p, int a) {
  AxisTables& t = p->ax[a];
  t.n = p->n[a];
  t.N = t.n - 1;
  t.scale = 2.0 / (p->hi[a] - p->lo[a]);
  t.transform_ok = t.N >= 2 && t.N <= kTransformMaxN;
  t.chirp = !(is_pow2(t.N) && t.N >= 4);
  t.dense_ok = t.n <= kDenseMaxN;
  t.route = line_route(t);
  t.route32 = t.route;
  if (t.transform_ok) {
    t.P = t.chirp ? std::max(8, next_pow2(4 * t.N - 1)) : 2 * t.N;
    // per-stage twiddles of the warp FFT (radix 8, then 4 or 2):
    // stage with span Ns and radix R stores exp(-2 pi i r k / (Ns R)) at
    // (Ns - 1) + (r - 1) Ns + k, r = 1..R-1, k < Ns
    std::vector<double2> tw64(t.P, make_double2(1.0, 0.0));
    std::vector<float2> tw32(t.P, make_float2(1.f, 0.f));
    for (int Ns = 1, rem = t.P; rem > 1;) {
      const int R = rem % 8 == 0 ? 8 : rem;
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          const double ang = -2.0 * M_PI * (double)(r * k) / (double)(Ns * R);
          const int at = (Ns - 1) + (r - 1) * Ns + k;
          tw64[at] = make_double2(std::cos(ang), std::sin(ang));
          tw32[at] = make_float2((float)tw64[at].x, (float)tw64[at].y);
        }
      Ns *= R;
      rem /= R;
    }
    CHEB_CUDA(cudaMalloc(&t.tw64, sizeof(double2) * t.P));
    CHEB_CUDA(cudaMalloc(&t.tw32, sizeof(float2) * t.P));
    CHEB_CUDA(cudaMemcpy(t.tw64, tw64.data(), sizeof(double2) * t.P, cudaMemcpyHostToDevice));
    CHEB_CUDA(cudaMemcpy(t.tw32, tw32.data(), sizeof(float2) * t.P, cudaMemcpyHostToDevice));
    if (t.chirp) {
      std::vector<double2> c64, b64;
      chirp_tables(t.N, t.P, c64, b64);
      std::vector<float2> c32(c64.size()), b32(b64.size());
      for (size_t i = 0; i < c64.size(); ++i) c32[i] = make_float2((float)c64[i].x, (float)c64[i].y);
      for (size_t i = 0; i < b64.size(); ++i) b32[i] = make_float2((float)b64[i].x, (float)b64[i].y);
      CHEB_CUDA(cudaMalloc(&t.chirp64, sizeof(double2) * c64.size()));
      CHEB_CUDA(cudaMalloc(&t.chirp32, sizeof(float2) * c32.size()));
      CHEB_CUDA(cudaMalloc(&t.bhat64, sizeof(double2) * b64.size()));
      CHEB_CUDA(cudaMalloc(&t.bhat32, sizeof(float2) * b32.size()));
      CHEB_CUDA(cudaMemcpy(t.chirp64, c64.data(), sizeof(double2) * c64.size(), cudaMemcpyHostToDevice));
      CHEB_CUDA(cudaMemcpy(t.chirp32, c32.data(), sizeof(float2) * c32.size(), cudaMemcpyHostToDevice));
      CHEB_CUDA(cudaMemcpy(t.bhat64, b64.data(), sizeof(double2) * b64.size(), cudaMemcpyHostToDevice));
      CHEB_CUDA(cudaMemcpy(t.bhat32, b32.data(), sizeof(float2) * b32.size(), cudaMemcpyHostToDevice));
    }
  }
  if (t.dense_ok) {
    std::vector<double> D = dense_deriv_matrix(t.N, t.scale);
    std::vector<float> D32(D.size());
    for (size_t i = 0; i < D.size(); ++i) D32[i] = (float)D[i];
    CHEB_CUDA(cudaMalloc(&t.D64, sizeof(double) * D.size()));
    CHEB_CUDA(cudaMalloc(&t.D32, sizeof(float) * D.size()));
    CHEB_CUDA(cudaMemcpy(t.D64, D.data(), sizeof(double) * D.size(), cudaMemcpyHostToDevice));
    CHEB_CUDA(cudaMemcpy(t.D32, D32.data(), sizeof(float) * D.size(), cudaMemcpyHostToDevice));
  }
  if (!t.transform_ok && !t.dense_ok) {
    set_error("axis size supported by neither route");
    return CHEB_ERR_UNSUPPORTED;
  }
  {
    const std::vector<double> w = cc_weights(t.N, 0.5 * (p->hi[a] - p->lo[a]));
    CHEB_CUDA(cudaMalloc(&t.cc64, sizeof(double) * w.size()));
    CHEB_CUDA(cudaMemcpy(t.cc64, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice));
  }
  return CHEB_OK;
}

static void free_axis(AxisTables& t) {
  cudaFree(t.tw64); cudaFree(t.tw32); cudaFree(t.D64); cudaFree(t.D32); cudaFree(t.cc64);
  cudaFree(t.chirp64); cudaFree(t.chirp32); cudaFree(t.bhat64); cudaFree(t.bhat32);
  t.tw64 = nullptr; t.tw32 = nullptr; t.D64 = nullptr; t.D32 = nullptr; t.cc64 = nullptr;
  t.chirp64 = nullptr; t.chirp32 = nullptr; t.bhat64 = nullptr; t.bhat32 = nullptr;
}

}  // namespace cheb

using namespace cheb;

extern "C" {

const char* cheb_last_error(void) { return g_last_error.c_str(); }

long long cheb_launch_count(void) { return g_launches.load(); }

int cheb_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  collect_locked();
  for (int c = 0; c < kProfNCat; ++c) { g_prof.ms[c] = 0.0; g_prof.cnt[c] = 0; g_prof.open[c] = nullptr; }
  g_prof.on = on != 0;
  return CHEB_OK;
}

int cheb_profile_read(double* ms, long long* counts) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  collect_locked();
  for (int c = 0; c < kProfNCat; ++c) {
    if (ms) ms[c] = g_prof.ms[c];
    if (counts) counts[c] = g_prof.cnt[c];
  }
  return CHEB_OK;
}

const char* cheb_status_str(int status) {
  switch (status) {
    case CHEB_OK: return "ok";
    case CHEB_ERR_NOT_CONVERGED: return "not converged";
    case CHEB_ERR_ARG: return "invalid argument";
    case CHEB_ERR_CUDA: return "CUDA error";
    case CHEB_ERR_NOMEM: return "out of device memory";
    case CHEB_ERR_NONFINITE: return "non-finite residual";
    case CHEB_ERR_SINGULAR_BC: return "singular boundary conditions (no Dirichlet face)";
    case CHEB_ERR_UNSUPPORTED: return "unsupported size or route";
    default: return "unknown status";
  }
}

int cheb_plan_create(cheb_plan* out, int dim, const int n[3], const double lo[3],
                     const double hi[3], const int bc_type[6], void* stream) {
  if (!out || !n || !lo || !hi || !bc_type) { set_error("null argument"); return CHEB_ERR_ARG; }
  *out = nullptr;
  if (dim < 1 || dim > 3) { set_error("dim must be 1, 2 or 3"); return CHEB_ERR_ARG; }
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      if (n[a] < 3) { set_error("active axes need n >= 3"); return CHEB_ERR_ARG; }
      if (!(hi[a] > lo[a]) || !std::isfinite(hi[a] - lo[a])) {
        set_error("need hi > lo"); return CHEB_ERR_ARG;
      }
    } else if (n[a] != 1) { set_error("unused axes need n = 1"); return CHEB_ERR_ARG; }
  }
  for (int f = 0; f < 6; ++f)
    if (bc_type[f] != CHEB_DIRICHLET && bc_type[f] != CHEB_NEUMANN && bc_type[f] != CHEB_FLUX) {
      set_error("bc_type must be CHEB_DIRICHLET, CHEB_NEUMANN or CHEB_FLUX"); return CHEB_ERR_ARG;
    }
  cheb_plan_s* p = new cheb_plan_s();
  p->dim = dim;
  for (int a = 0; a < 3; ++a) {
    p->n[a] = n[a];
    p->lo[a] = a < dim ? lo[a] : -1.0;
    p->hi[a] = a < dim ? hi[a] : 1.0;
  }
  for (int f = 0; f < 6; ++f) p->bc[f] = bc_type[f];
  p->stream = (cudaStream_t)stream;
  cudaGetDevice(&p->device);
  for (int a = 0; a < dim; ++a) {
    int st = build_axis(p, a);
    if (st != CHEB_OK) { cheb_plan_destroy(p); return st; }
  }
  *out = p;
  return CHEB_OK;
}

int cheb_plan_destroy(cheb_plan p) {
  if (!p) return CHEB_OK;
  free_workspace(p);
  tensor_apply_free(p->tap);
  p->tap = nullptr;
  for (int a = 0; a < 3; ++a) free_axis(p->ax[a]);
  delete p;
  return CHEB_OK;
}

int cheb_plan_set_stream(cheb_plan p, void* stream) {
  if (!p) return CHEB_ERR_ARG;
  p->stream = (cudaStream_t)stream;
  return CHEB_OK;
}

int cheb_plan_set_route(cheb_plan p, int axis, int route) {
  if (!p || axis < 0 || axis >= p->dim) { set_error("bad plan or axis"); return CHEB_ERR_ARG; }
  AxisTables& t = p->ax[axis];
  if (route == CHEB_ROUTE_AUTO) route = line_route(t);
  if (route == CHEB_ROUTE_TRANSFORM && !t.transform_ok) {
    set_error("transform route needs 2 <= n - 1 <= 256"); return CHEB_ERR_UNSUPPORTED;
  }
  if (route == CHEB_ROUTE_DENSE && !t.dense_ok) {
    set_error("dense route needs n <= 129"); return CHEB_ERR_UNSUPPORTED;
  }
  if (route != CHEB_ROUTE_TRANSFORM && route != CHEB_ROUTE_DENSE) {
    set_error("unknown route"); return CHEB_ERR_ARG;
  }
  t.route = route;
  t.route32 = route;
  return CHEB_OK;
}

int cheb_plan_set_route32(cheb_plan p, int axis, int route) {
  if (!p || axis < 0 || axis >= p->dim) { set_error("bad plan or axis"); return CHEB_ERR_ARG; }
  AxisTables& t = p->ax[axis];
  if (route == CHEB_ROUTE_AUTO) route = line_route(t);
  if (route == CHEB_ROUTE_TRANSFORM && !t.transform_ok) {
    set_error("transform route needs 2 <= n - 1 <= 256"); return CHEB_ERR_UNSUPPORTED;
  }
  if (route == CHEB_ROUTE_DENSE && !t.dense_ok) {
    set_error("dense route needs n <= 129"); return CHEB_ERR_UNSUPPORTED;
  }
  if (route == CHEB_ROUTE_TENSOR && !tensor_route_ok(p, axis)) {
    set_error("tensor route needs a 2-D or 3-D grid, 33 <= n <= 257, at least 128 lines and no flux face");
    return CHEB_ERR_UNSUPPORTED;
  }
  if (route != CHEB_ROUTE_TRANSFORM && route != CHEB_ROUTE_DENSE && route != CHEB_ROUTE_TENSOR) {
    set_error("unknown route"); return CHEB_ERR_ARG;
  }
  t.route32 = route;
  return CHEB_OK;
}

int cheb_plan_set_tile(cheb_plan p, int axis, int prec, int lines) {
  if (!p || axis < 0 || axis >= p->dim) { set_error("bad plan or axis"); return CHEB_ERR_ARG; }
  if (lines != 8 && lines != 16) { set_error("line tiles of 8 or 16 lines"); return CHEB_ERR_ARG; }
  if (prec == CHEB_FP64) p->ax[axis].tile = lines;
  else if (prec == CHEB_FP32) p->ax[axis].tile32 = lines;
  else { set_error("prec must be CHEB_FP64 or CHEB_FP32"); return CHEB_ERR_ARG; }
  return CHEB_OK;
}

int cheb_plan_get_tile(cheb_plan p, int axis, int prec, int* lines) {
  if (!p || !lines || axis < 0 || axis >= p->dim) { set_error("bad argument"); return CHEB_ERR_ARG; }
  if (prec == CHEB_FP64) *lines = p->ax[axis].tile;
  else if (prec == CHEB_FP32) *lines = p->ax[axis].tile32;
  else { set_error("prec must be CHEB_FP64 or CHEB_FP32"); return CHEB_ERR_ARG; }
  return CHEB_OK;
}

int cheb_plan_get_route32(cheb_plan p, int axis, int* route) {
  if (!p || !route || axis < 0 || axis >= p->dim) { set_error("bad argument"); return CHEB_ERR_ARG; }
  *route = p->ax[axis].route32;
  return CHEB_OK;
}

int cheb_plan_get_route(cheb_plan p, int axis, int* route) {
  if (!p || !route || axis < 0 || axis >= p->dim) { set_error("bad argument"); return CHEB_ERR_ARG; }
  *route = p->ax[axis].route;
  return CHEB_OK;
}

size_t cheb_plan_size(cheb_plan p) { return p ? p->size() : 0; }

int cheb_nodes(cheb_plan p, int axis, double* out) {
  if (!p || !out || axis < 0 || axis > 2) { set_error("bad argument"); return CHEB_ERR_ARG; }
  if (axis >= p->dim) { out[0] = 0.0; return CHEB_OK; }
  const int N = p->n[axis] - 1;
  const double h = 0.5 * (p->hi[axis] - p->lo[axis]), c = 0.5 * (p->hi[axis] + p->lo[axis]);
  for (int j = 0; j <= N; ++j) out[j] = h * cgl_ref(j, N) + c;
  return CHEB_OK;
}

int cheb_deriv(cheb_plan p, int prec, int axis, const void* u, void* du) {
  if (!p || !u || !du || axis < 0 || axis >= p->dim) { set_error("bad argument"); return CHEB_ERR_ARG; }
  if (prec == CHEB_FP64)
    return launch_pass<double>(p, axis, kDeriv, nullptr, (const double*)u, (double*)du, p->stream);
  if (prec == CHEB_FP32)
    return launch_pass<float>(p, axis, kDeriv, nullptr, (const float*)u, (float*)du, p->stream);
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}

int cheb_deriv_t(cheb_plan p, int prec, int axis, const void* u, void* du) {
  if (!p || !u || !du || axis < 0 || axis >= p->dim) { set_error("bad argument"); return CHEB_ERR_ARG; }
  if (prec == CHEB_FP64)
    return launch_pass<double>(p, axis, kDerivT, nullptr, (const double*)u, (double*)du, p->stream);
  if (prec == CHEB_FP32)
    return launch_pass<float>(p, axis, kDerivT, nullptr, (const float*)u, (float*)du, p->stream);
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}

int cheb_apply(cheb_plan p, int prec, const void* K, const void* u, void* Au) {
  if (!p || !K || !u || !Au) { set_error("null argument"); return CHEB_ERR_ARG; }
  if (Au == u || Au == K) { set_error("Au must not alias K or u"); return CHEB_ERR_ARG; }
  if (prec == CHEB_FP64)
    return launch_apply<double>(p, (const double*)K, (const double*)u, (double*)Au, p->stream);
  if (prec == CHEB_FP32)
    return launch_apply<float>(p, (const float*)K, (const float*)u, (float*)Au, p->stream);
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}

int cheb_adjoint_apply(cheb_plan p, int prec, const void* K, const void* lam, void* ATlam) {
  if (!p || !K || !lam || !ATlam) { set_error("null argument"); return CHEB_ERR_ARG; }
  if (ATlam == lam || ATlam == K) { set_error("output must not alias K or lam"); return CHEB_ERR_ARG; }
  if (prec == CHEB_FP64)
    return launch_adjoint_apply<double>(p, (const double*)K, (const double*)lam, (double*)ATlam, p->stream);
  if (prec == CHEB_FP32)
    return launch_adjoint_apply<float>(p, (const float*)K, (const float*)lam, (float*)ATlam, p->stream);
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}

int cheb_rhs(cheb_plan p, const double* f, const double* const face_vals[6], double* b) {
  if (!p || !f || !b || !face_vals) { set_error("null argument"); return CHEB_ERR_ARG; }
  for (int fc = 0; fc < 2 * p->dim; ++fc)
    if (!face_vals[fc]) { set_error("null face array of an active axis"); return CHEB_ERR_ARG; }
  const double* fv[6];
  for (int fc = 0; fc < 6; ++fc) fv[fc] = fc < 2 * p->dim ? face_vals[fc] : f;
  return launch_rhs(p, f, fv, b, p->stream);
}

}  // extern "C"
