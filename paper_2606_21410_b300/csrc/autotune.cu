// Route autotuner: for every active axis and both precisions, time the
// operator line pass on the plan's own grid with every route the axis size
// allows - the FFT transform route and the dense differentiation-matrix route,
// each with line tiles of 8 and of 16 lines per CTA, and for FP32 the
// tensor-core route - and keep the fastest (route, tile).  Decisions are
// cached in a plain text file, one line per (GPU name, axis size, precision),
// so later plans of the same size skip the timing.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "umma.h"

namespace cheb {

namespace {
std::mutex g_tune_mu;

struct TuneRec {
  std::string gpu;
  int n = 0, bits = 0, route = 0, tile = 16;
  double ms_tf = 0, ms_dense = 0, ms_tensor = 0;  // best time of each route (0: not timed)
};

std::vector<TuneRec> load_cache(const char* path) {
  std::vector<TuneRec> v;
  if (!path) return v;
  FILE* f = std::fopen(path, "r");
  if (!f) return v;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    char gpu[256];
    TuneRec r;
    // format: "<gpu name with underscores> <n> <bits> <route> <tile> <ms_tf> <ms_dense> <ms_tensor>"
    if (std::sscanf(line, "%255s %d %d %d %d %lf %lf %lf", gpu, &r.n, &r.bits, &r.route, &r.tile, &r.ms_tf,
                    &r.ms_dense, &r.ms_tensor) == 8) {
      r.gpu = gpu;
      v.push_back(r);
    }
  }
  std::fclose(f);
  return v;
}

void append_cache(const char* path, const TuneRec& r) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d %.6f %.6f %.6f\n", r.gpu.c_str(), r.n, r.bits, r.route, r.tile, r.ms_tf,
               r.ms_dense, r.ms_tensor);
  std::fclose(f);
}

std::string gpu_key() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string s = prop.name;
  for (auto& c : s)
    if (c == ' ') c = '_';
  return s;
}

template <typename T>
int time_pass(cheb_plan_s* p, int axis, T* K, T* u, T* out, float* ms) {
  cudaEvent_t a, b;
  CHEB_CUDA(cudaEventCreate(&a));
  CHEB_CUDA(cudaEventCreate(&b));
  int st = CHEB_OK;
  for (int r = 0; r < 2 && !st; ++r) st = launch_pass<T>(p, axis, kApplyAcc, K, u, out, p->stream);
  CHEB_CUDA(cudaEventRecord(a, p->stream));
  const int reps = 5;
  for (int r = 0; r < reps && !st; ++r) st = launch_pass<T>(p, axis, kApplyAcc, K, u, out, p->stream);
  CHEB_CUDA(cudaEventRecord(b, p->stream));
  CHEB_CUDA(cudaEventSynchronize(b));
  float t = 0;
  cudaEventElapsedTime(&t, a, b);
  *ms = t / reps;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

// (route, tile) pairs the axis allows in this precision
struct Cand { int route, tile; };
template <typename T>
std::vector<Cand> candidates(const cheb_plan_s* p, int a) {
  std::vector<Cand> c;
  const AxisTables& t = p->ax[a];
  for (int tile : {16, 8}) {
    // the chirp form of the transform route always runs 8-line tiles
    if (t.transform_ok && (!t.chirp || tile == 8)) c.push_back({CHEB_ROUTE_TRANSFORM, tile});
    if (t.dense_ok) c.push_back({CHEB_ROUTE_DENSE, tile});
  }
  if (sizeof(T) == 4 && tensor_route_ok(p, a)) c.push_back({CHEB_ROUTE_TENSOR, 16});
  return c;
}

template <typename T>
int tune_precision(cheb_plan_s* p, const char* cache, const std::string& gpu, int* routes_out) {
  const size_t n = p->size();
  T *K = nullptr, *u = nullptr, *out = nullptr;
  const int bits = (int)sizeof(T) * 8;
  std::vector<TuneRec> cached = load_cache(cache);
  bool need = false;
  for (int a = 0; a < p->dim; ++a) {
    const AxisTables& t = p->ax[a];
    if (candidates<T>(p, a).size() < 2) continue;
    bool hit = false;
    for (auto& r : cached)
      if (r.gpu == gpu && r.n == t.n && r.bits == bits) hit = true;
    need |= !hit;
  }
  if (need) {
    CHEB_CUDA(cudaMalloc(&K, sizeof(T) * n));
    CHEB_CUDA(cudaMalloc(&u, sizeof(T) * n));
    CHEB_CUDA(cudaMalloc(&out, sizeof(T) * n));
    CHEB_CUDA(cudaMemsetAsync(K, 0, sizeof(T) * n, p->stream));
    CHEB_CUDA(cudaMemsetAsync(u, 0, sizeof(T) * n, p->stream));
    CHEB_CUDA(cudaMemsetAsync(out, 0, sizeof(T) * n, p->stream));
  }
  int st = CHEB_OK;
  for (int a = 0; a < p->dim && !st; ++a) {
    AxisTables& t = p->ax[a];
    int& route = (sizeof(T) == 4) ? t.route32 : t.route;
    int& tile = (sizeof(T) == 4) ? t.tile32 : t.tile;
    const std::vector<Cand> cand = candidates<T>(p, a);
    if (cand.size() < 2) {
      routes_out[a] = route;
      continue;
    }
    const TuneRec* hit = nullptr;
    for (auto& r : cached)
      if (r.gpu == gpu && r.n == t.n && r.bits == bits) hit = &r;
    if (hit) {
      route = hit->route;
      tile = hit->tile;
    } else {
      TuneRec r;
      float best = 0;
      Cand best_c = cand[0];
      bool first = true;
      for (const Cand& c : cand) {
        float ms = 0;
        route = c.route;
        tile = c.tile;
        if ((st = time_pass<T>(p, a, K, u, out, &ms))) break;
        double& slot = c.route == CHEB_ROUTE_TRANSFORM ? r.ms_tf : c.route == CHEB_ROUTE_DENSE ? r.ms_dense
                                                                                                : r.ms_tensor;
        if (slot == 0 || ms < slot) slot = ms;
        if (first || ms < best) { best = ms; best_c = c; first = false; }
      }
      if (st) break;
      route = best_c.route;
      tile = best_c.tile;
      r.gpu = gpu; r.n = t.n; r.bits = bits; r.route = route; r.tile = tile;
      append_cache(cache, r);
      cached.push_back(r);
    }
    routes_out[a] = route;
  }
  cudaFree(K); cudaFree(u); cudaFree(out);
  return st;
}

}  // namespace

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_autotune(cheb_plan p, const char* cache_path, int routes_out[6]) {
  if (!p) { set_error("null plan"); return CHEB_ERR_ARG; }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const std::string gpu = gpu_key();
  int r64[3] = {0, 0, 0}, r32[3] = {0, 0, 0};
  int st = tune_precision<double>(p, cache_path, gpu, r64);
  if (!st) st = tune_precision<float>(p, cache_path, gpu, r32);
  if (routes_out)
    for (int a = 0; a < 3; ++a) {
      routes_out[a] = r64[a];
      routes_out[3 + a] = r32[a];
    }
  return st;
}
