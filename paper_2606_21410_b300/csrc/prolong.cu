// Modal prolongation N -> 2N (Sec. 2.3.3, Alg. 4): per axis and per line,
// coarse nodal values -> Chebyshev coefficients a_k = c_k DCT-I(f)_k / N,
// zero-padding to degree 2N, and evaluation at the fine CGL nodes
// f_fine(x_n) = sum_{k<=N} a_k cos(pi k n / 2N) = DCT-I_{2N}(beta)_n with
// beta_0 = a_0, beta_k = a_k / 2 (1 <= k <= N, k = N is an interior mode of
// the fine transform), beta_k = 0 beyond.  Both transforms are warp FFTs of
// the even extensions (lengths P = 2N and 2P), two lines per complex FFT.
// Three axis passes, x then y then z, through two scratch arrays.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>


#include "device.cuh"
#include "fdm.h"
#include "krylov.h"
#include "prolong.h"

namespace cheb {

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename T, int PC>
static size_t prolong_smem() {
  const int nc = PC / 2 + 1;
  const int nf = 2 * (nc - 1) + 1;
  const int ldx = nf | 1;
  return al16(sizeof(T) * kTileL * ldx) + al16(2 * sizeof(T) * (size_t)(kTileL / 2) * FftBuf<2 * PC>::len) +
         al16(2 * sizeof(T) * (size_t)3 * PC);
}

// dims: extents of the input array (axis a has nc points); the output has
// 2(nc-1)+1 points along a.
template <typename T, int PC>
__global__ void __launch_bounds__(kThreads)
prolong_pass_kernel(int a, int nx, int ny, int nz, const typename C2<T>::t* __restrict__ twc,
                    const typename C2<T>::t* __restrict__ twf, const T* __restrict__ in,
                    T* __restrict__ out) {
  typedef typename C2<T>::t C;
  constexpr int NC = PC / 2;         // coarse N
  constexpr int PF = 2 * PC;         // fine FFT length
  constexpr int NF = 2 * NC;         // fine N
  const int nc = NC + 1, nf = NF + 1;
  const int ldx = nf | 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int BL = FftBuf<PF>::len;
  unsigned char* p = smem_raw;
  T* X = (T*)p;      p += al16(sizeof(T) * kTileL * ldx);
  C* Cb = (C*)p;     p += al16(2 * sizeof(T) * (size_t)(kTileL / 2) * BL);
  C* tw = (C*)p;     // fine-transform stage twiddles (PF), then coarse ones (PC)
  C* twc_s = tw + PF;
  for (int t = threadIdx.x; t < PF; t += blockDim.x) tw[t] = twf[t];
  for (int t = threadIdx.x; t < PC; t += blockDim.x) twc_s[t] = twc[t];
  // tile geometry: lines are indexed by the two other axes
  const int dims_in[3] = {nx, ny, nz};
  int dims_out[3] = {nx, ny, nz};
  dims_out[a] = nf;
  int line0 = 0, i0 = 0, outer = 0;
  if (a == 0) line0 = blockIdx.x * kTileL;
  else {
    const int nbx = (nx + kTileL - 1) / kTileL;
    i0 = (blockIdx.x % nbx) * kTileL;
    outer = blockIdx.x / nbx;
  }
  auto gidx = [&](const int* dims, int l, int pt, size_t& g) -> bool {
    if (a == 0) {
      const int line = line0 + l;
      if (line >= dims[1] * dims[2]) return false;
      g = (size_t)line * dims[0] + pt;
    } else {
      const int i = i0 + l;
      if (i >= dims[0]) return false;
      int j, k;
      if (a == 1) { j = pt; k = outer; } else { j = outer; k = pt; }
      g = ((size_t)k * dims[1] + j) * dims[0] + i;
    }
    return true;
  };
  for (int e = threadIdx.x; e < kTileL * nc; e += blockDim.x) {
    int l, pt;
    if (a == 0) { l = e / nc; pt = e - l * nc; } else { pt = e / kTileL; l = e - pt * kTileL; }
    size_t g;
    X[l * ldx + pt] = gidx(dims_in, l, pt, g) ? in[g] : (T)0;
  }
  __syncthreads();
  {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* xa = X + (2 * w) * ldx;
    T* xb = X + (2 * w + 1) * ldx;
    C* buf = Cb + (size_t)w * BL;
    // coarse DCT-I with the length-PC FFT
    for (int j = lane; j < PC; j += 32) {
      const int jj = j <= NC ? j : PC - j;
      C v; v.x = xa[jj]; v.y = xb[jj];
      buf[fpad(j)] = v;
    }
    __syncwarp();
    warp_fft<T, PC>(buf, twc_s, lane);
    // beta_k = F_k / (2 NC) for k < NC, F_NC / (4 NC); zero for k > NC
    const T s = (T)1 / (T)(2 * NC);
    for (int k = lane; k <= NF; k += 32) {
      T ba = 0, bb = 0;
      if (k <= NC) {
        const C F = buf[fpad(k)];
        const T wk = (k == NC) ? (T)0.5 * s : s;
        ba = wk * F.x;
        bb = wk * F.y;
      }
      xa[k] = ba;
      xb[k] = bb;
    }
    __syncwarp();
    for (int j = lane; j < PF; j += 32) {
      const int jj = j <= NF ? j : PF - j;
      C v; v.x = xa[jj]; v.y = xb[jj];
      buf[fpad(j)] = v;
    }
    __syncwarp();
    warp_fft<T, PF>(buf, tw, lane);
    for (int k = lane; k <= NF; k += 32) {
      const C F = buf[fpad(k)];
      xa[k] = F.x;
      xb[k] = F.y;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kTileL * nf; e += blockDim.x) {
    int l, pt;
    if (a == 0) { l = e / nf; pt = e - l * nf; } else { pt = e / kTileL; l = e - pt * kTileL; }
    size_t g;
    if (gidx(dims_out, l, pt, g)) out[g] = X[l * ldx + pt];
  }
}

template <typename T, int PC>
static int launch_prolong_pass(int a, const int dims[3], const typename C2<T>::t* twc,
                               const typename C2<T>::t* twf, const T* in, T* out, cudaStream_t s) {
  auto kern = prolong_pass_kernel<T, PC>;
  const size_t smem = prolong_smem<T, PC>();
  int st;
  if ((st = ensure_smem_attr((const void*)kern, smem))) return st;
  int nblocks;
  if (a == 0) nblocks = (dims[1] * dims[2] + kTileL - 1) / kTileL;
  else nblocks = ((dims[0] + kTileL - 1) / kTileL) * (a == 1 ? dims[2] : dims[1]);
  kern<<<nblocks, kThreads, smem, s>>>(a, dims[0], dims[1], dims[2], twc, twf, in, out);
  CHEB_LAUNCH_CHECK("prolong_pass_kernel");
  return CHEB_OK;
}

// ---------------------------------------------------------------------------
// Chirp form (coarse N not a power of two, so neither is the fine 2N): both
// DCT-Is are length-2N / 4N DFTs by Bluestein's convolution, FFT lengths LC
// and LF = 2 LC (nextpow2(8N - 1) = 2 nextpow2(4N - 1): neither 8N - 1 nor
// 8N - 2 is a power of two).  Eight-line tiles, one line pair per warp.
// ---------------------------------------------------------------------------
template <typename T>
struct ChirpTabs {
  const typename C2<T>::t* tw;     // stage twiddles (L)
  const typename C2<T>::t* chirp;  // c_j, j < M
  const typename C2<T>::t* bhat;   // transformed kernel (L)
};
constexpr int kChirpTileL = 8;

template <typename T, int LC>
static size_t prolong_chirp_smem(int nf) {
  constexpr int LF = 2 * LC;
  const int ldx = nf | 1;
  return al16(sizeof(T) * kChirpTileL * ldx) +
         al16(2 * sizeof(T) * (size_t)(kChirpTileL / 2) * FftBuf<LF>::len) +
         al16(2 * sizeof(T) * (size_t)(LF + LF / 2 + LF)) + al16(2 * sizeof(T) * (size_t)(LC + LC / 2 + LC));
}

template <typename T, int LC>
__global__ void __launch_bounds__(kChirpTileL * 16)
prolong_chirp_kernel(int a, int nx, int ny, int nz, int NC, ChirpTabs<T> tc, ChirpTabs<T> tf,
                     const T* __restrict__ in, T* __restrict__ out) {
  typedef typename C2<T>::t C;
  constexpr int LF = 2 * LC;
  constexpr int TLn = kChirpTileL;
  const int NF = 2 * NC, MC = 2 * NC, MF = 2 * NF;
  const int nc = NC + 1, nf = NF + 1;
  const int ldx = nf | 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int BL = FftBuf<LF>::len;
  unsigned char* p = smem_raw;
  T* X = (T*)p;   p += al16(sizeof(T) * TLn * ldx);
  C* Cb = (C*)p;  p += al16(2 * sizeof(T) * (size_t)(TLn / 2) * BL);
  C* twf = (C*)p; C* chf = twf + LF; C* bhf = chf + LF / 2;
  p += al16(2 * sizeof(T) * (size_t)(LF + LF / 2 + LF));
  C* twc = (C*)p; C* chc = twc + LC; C* bhc = chc + LC / 2;
  for (int t = threadIdx.x; t < LF; t += blockDim.x) { twf[t] = tf.tw[t]; bhf[t] = tf.bhat[t]; }
  for (int t = threadIdx.x; t < MF; t += blockDim.x) chf[t] = tf.chirp[t];
  for (int t = threadIdx.x; t < LC; t += blockDim.x) { twc[t] = tc.tw[t]; bhc[t] = tc.bhat[t]; }
  for (int t = threadIdx.x; t < MC; t += blockDim.x) chc[t] = tc.chirp[t];
  const int dims_in[3] = {nx, ny, nz};
  int dims_out[3] = {nx, ny, nz};
  dims_out[a] = nf;
  int line0 = 0, i0 = 0, outer = 0;
  if (a == 0) line0 = blockIdx.x * TLn;
  else {
    const int nbx = (nx + TLn - 1) / TLn;
    i0 = (blockIdx.x % nbx) * TLn;
    outer = blockIdx.x / nbx;
  }
  auto gidx = [&](const int* dims, int l, int pt, size_t& g) -> bool {
    if (a == 0) {
      const int line = line0 + l;
      if (line >= dims[1] * dims[2]) return false;
      g = (size_t)line * dims[0] + pt;
    } else {
      const int i = i0 + l;
      if (i >= dims[0]) return false;
      int j, k;
      if (a == 1) { j = pt; k = outer; } else { j = outer; k = pt; }
      g = ((size_t)k * dims[1] + j) * dims[0] + i;
    }
    return true;
  };
  for (int e = threadIdx.x; e < TLn * nc; e += blockDim.x) {
    int l, pt;
    if (a == 0) { l = e / nc; pt = e - l * nc; } else { pt = e / TLn; l = e - pt * TLn; }
    size_t g;
    X[l * ldx + pt] = gidx(dims_in, l, pt, g) ? in[g] : (T)0;
  }
  __syncthreads();
  {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* xa = X + (2 * w) * ldx;
    T* xb = X + (2 * w + 1) * ldx;
    C* buf = Cb + (size_t)w * BL;
    // coarse DCT-I: length-2NC DFT of the even extension
    for (int j = lane; j < MC; j += 32) {
      const int jj = j <= NC ? j : MC - j;
      C v; v.x = xa[jj]; v.y = xb[jj];
      buf[fpad(j)] = v;
    }
    __syncwarp();
    warp_dft_chirp<T, LC>(buf, twc, chc, bhc, MC, lane);
    // beta_k = F_k / (2 NC) for k < NC, F_NC / (4 NC); zero for k > NC
    const T s = (T)1 / (T)(2 * NC);
    for (int k = lane; k <= NF; k += 32) {
      T ba = 0, bb = 0;
      if (k <= NC) {
        const C F = buf[fpad(k)];
        const T wk = (k == NC) ? (T)0.5 * s : s;
        ba = wk * F.x;
        bb = wk * F.y;
      }
      xa[k] = ba;
      xb[k] = bb;
    }
    __syncwarp();
    // fine DCT-I: length-2NF DFT of the padded coefficients' even extension
    for (int j = lane; j < MF; j += 32) {
      const int jj = j <= NF ? j : MF - j;
      C v; v.x = xa[jj]; v.y = xb[jj];
      buf[fpad(j)] = v;
    }
    __syncwarp();
    warp_dft_chirp<T, LF>(buf, twf, chf, bhf, MF, lane);
    for (int k = lane; k <= NF; k += 32) {
      const C F = buf[fpad(k)];
      xa[k] = F.x;
      xb[k] = F.y;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TLn * nf; e += blockDim.x) {
    int l, pt;
    if (a == 0) { l = e / nf; pt = e - l * nf; } else { pt = e / TLn; l = e - pt * TLn; }
    size_t g;
    if (gidx(dims_out, l, pt, g)) out[g] = X[l * ldx + pt];
  }
}

template <typename T, int LC>
static int launch_prolong_chirp(int a, const int dims[3], int NC, const ChirpTabs<T>& tc, const ChirpTabs<T>& tf,
                                const T* in, T* out, cudaStream_t s) {
  auto kern = prolong_chirp_kernel<T, LC>;
  const size_t smem = prolong_chirp_smem<T, LC>(2 * NC + 1);
  int st;
  if ((st = ensure_smem_attr((const void*)kern, smem))) return st;
  int nblocks;
  if (a == 0) nblocks = (dims[1] * dims[2] + kChirpTileL - 1) / kChirpTileL;
  else nblocks = ((dims[0] + kChirpTileL - 1) / kChirpTileL) * (a == 1 ? dims[2] : dims[1]);
  if (nblocks == 0) return CHEB_OK;
  kern<<<nblocks, kChirpTileL * 16, smem, s>>>(a, dims[0], dims[1], dims[2], NC, tc, tf, in, out);
  CHEB_LAUNCH_CHECK("prolong_chirp_kernel");
  return CHEB_OK;
}

template <typename T> static ChirpTabs<T> chirp_tabs(const AxisTables& t);
template <> ChirpTabs<double> chirp_tabs<double>(const AxisTables& t) { return {t.tw64, t.chirp64, t.bhat64}; }
template <> ChirpTabs<float> chirp_tabs<float>(const AxisTables& t) { return {t.tw32, t.chirp32, t.bhat32}; }

template <typename T>
static int prolong_chirp_pass(int a, const AxisTables& c, const AxisTables& f, const int dims[3], const T* in,
                              T* out, cudaStream_t s) {
  const ChirpTabs<T> tc = chirp_tabs<T>(c), tf = chirp_tabs<T>(f);
  const int NC = c.N;
  switch (c.P) {
    case 16: return launch_prolong_chirp<T, 16>(a, dims, NC, tc, tf, in, out, s);
    case 32: return launch_prolong_chirp<T, 32>(a, dims, NC, tc, tf, in, out, s);
    case 64: return launch_prolong_chirp<T, 64>(a, dims, NC, tc, tf, in, out, s);
    case 128: return launch_prolong_chirp<T, 128>(a, dims, NC, tc, tf, in, out, s);
    case 256: return launch_prolong_chirp<T, 256>(a, dims, NC, tc, tf, in, out, s);
    case 512: return launch_prolong_chirp<T, 512>(a, dims, NC, tc, tf, in, out, s);
    default:
      set_error("chirp prolongation needs coarse convolution length in [16, 512]");
      return CHEB_ERR_UNSUPPORTED;
  }
}

template <typename T> static const typename C2<T>::t* twf_of(const AxisTables& t);
template <> const double2* twf_of<double>(const AxisTables& t) { return t.tw64; }
template <> const float2* twf_of<float>(const AxisTables& t) { return t.tw32; }

template <typename T>
static int prolong_pass(int a, int PC, const int dims[3], const typename C2<T>::t* twc,
                        const typename C2<T>::t* twf, const T* in, T* out, cudaStream_t s) {
  switch (PC) {
    case 8: return launch_prolong_pass<T, 8>(a, dims, twc, twf, in, out, s);
    case 16: return launch_prolong_pass<T, 16>(a, dims, twc, twf, in, out, s);
    case 32: return launch_prolong_pass<T, 32>(a, dims, twc, twf, in, out, s);
    case 64: return launch_prolong_pass<T, 64>(a, dims, twc, twf, in, out, s);
    case 128: return launch_prolong_pass<T, 128>(a, dims, twc, twf, in, out, s);
    case 256: return launch_prolong_pass<T, 256>(a, dims, twc, twf, in, out, s);
    default:
      set_error("prolongation needs coarse N a power of two in [4, 128]");
      return CHEB_ERR_UNSUPPORTED;
  }
}

int check_prolong_pair(const cheb_plan_s* c, const cheb_plan_s* f) {
  if (!c || !f || c->dim != f->dim) { set_error("plans must have the same dimension"); return CHEB_ERR_ARG; }
  for (int a = 0; a < c->dim; ++a) {
    if (f->n[a] - 1 != 2 * (c->n[a] - 1)) { set_error("fine N must be twice the coarse N"); return CHEB_ERR_ARG; }
    if (c->lo[a] != f->lo[a] || c->hi[a] != f->hi[a]) { set_error("plans must share the box"); return CHEB_ERR_ARG; }
    // power-of-two coarse N >= 4 (plain FFTs) or any coarse N >= 3 (chirp
    // form); the fine N is at most 256.  Coarse N = 2 (chirp) with fine
    // N = 4 (plain) mixes the two forms and is not supported.
    const AxisTables &ca = c->ax[a], &fa = f->ax[a];
    if (!fa.transform_ok || !ca.transform_ok || ca.chirp != fa.chirp || (ca.chirp && fa.P != 2 * ca.P)) {
      set_error("prolongation needs 3 <= coarse N and fine N = 2 coarse N <= 256");
      return CHEB_ERR_UNSUPPORTED;
    }
  }
  return CHEB_OK;
}

template <typename T>
int launch_prolong(const cheb_plan_s* c, const cheb_plan_s* f, const T* uc, T* uf, T* s1, T* s2,
                   cudaStream_t s) {
  int dims[3] = {c->n[0], c->n[1], c->n[2]};
  const T* src = uc;
  int st;
  for (int a = 0; a < c->dim; ++a) {
    T* dst = (a == c->dim - 1) ? uf : (a % 2 == 0 ? s1 : s2);
    if (c->ax[a].chirp) st = prolong_chirp_pass<T>(a, c->ax[a], f->ax[a], dims, src, dst, s);
    else st = prolong_pass<T>(a, 2 * (c->n[a] - 1), dims, twf_of<T>(c->ax[a]), twf_of<T>(f->ax[a]), src, dst, s);
    if (st) return st;
    dims[a] = f->n[a];
    src = dst;
  }
  return CHEB_OK;
}

template int launch_prolong<double>(const cheb_plan_s*, const cheb_plan_s*, const double*, double*, double*, double*, cudaStream_t);
template int launch_prolong<float>(const cheb_plan_s*, const cheb_plan_s*, const float*, float*, float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// Prolongation without allocation, for callers that cannot call cudaMalloc
// (for example code that runs inside a custom allocator, a memory-capped
// sandbox, or a process whose allocator must not be re-entered).  The two
// intermediate arrays of the axis passes live in one fixed file-scope device
// array of kNoAllocBytes; every GPU that loads this library holds it until
// the process exits.  The host code only knows the array by its symbol, so
// its device address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_prolong_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;
}  // namespace

static int noalloc_scratch(void** out) {
  int dev = 0;
  CHEB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) { set_error("device index out of range"); return CHEB_ERR_ARG; }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    CHEB_CUDA(cudaGetSymbolAddress(&ptr, g_prolong_scratch));
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return CHEB_OK;
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_prolong_noalloc(cheb_plan coarse, cheb_plan fine, int prec, const void* uc,
                                    void* uf) {
  if (!uc || !uf) { set_error("null argument"); return CHEB_ERR_ARG; }
  int st;
  if ((st = check_prolong_pair(coarse, fine))) return st;
  if (prec != CHEB_FP64 && prec != CHEB_FP32) {
    set_error("prec must be CHEB_FP64 or CHEB_FP32");
    return CHEB_ERR_ARG;
  }
  // intermediate extents: after the x pass (nxf, nyc, nzc), after the y pass (nxf, nyf, nzc)
  const size_t esz = prec == CHEB_FP64 ? sizeof(double) : sizeof(float);
  size_t n1 = 0, n2 = 0;
  if (coarse->dim >= 2) n1 = (size_t)fine->n[0] * coarse->n[1] * coarse->n[2];
  if (coarse->dim >= 3) n2 = (size_t)fine->n[0] * fine->n[1] * coarse->n[2];
  const size_t off2 = ((n1 * esz + 255) / 256) * 256;
  if (off2 + n2 * esz > kNoAllocBytes) {
    set_error("cheb_prolong_noalloc: the grids need " + std::to_string(off2 + n2 * esz) +
              " bytes of intermediate storage, above its fixed 16 MiB (use cheb_prolong)");
    return CHEB_ERR_UNSUPPORTED;
  }
  // the scratch address is per device: the plans' device must be current
  int dev = 0;
  CHEB_CUDA(cudaGetDevice(&dev));
  if (dev != coarse->device || dev != fine->device) {
    set_error("cheb_prolong_noalloc: the current device is not the plans' device");
    return CHEB_ERR_ARG;
  }
  void* base = nullptr;
  if ((st = noalloc_scratch(&base))) return st;
  unsigned char* b = (unsigned char*)base;
  if (prec == CHEB_FP64)
    return launch_prolong<double>(coarse, fine, (const double*)uc, (double*)uf, (double*)b,
                                  (double*)(b + off2), fine->stream);
  return launch_prolong<float>(coarse, fine, (const float*)uc, (float*)uf, (float*)b,
                               (float*)(b + off2), fine->stream);
}
