// Tensor-product contraction on the 5th-generation tensor cores (tcgen05).
//
// The fast-diagonalization preconditioner applies S^{-1} and S along each
// axis of the compact interior array: a dense (m_a x m_a) matrix against
// every a-line.  Contracting along the contiguous axis and writing the
// result transposed ([n][rows]) rotates the axes (x,y,z) -> (y,z,x), so three
// consecutive contractions return to the original layout and every operand
// is K-major: X rows (lines) as the MMA A operand, the matrix rows as B.
//
// Per CTA: 128 lines (UMMA M = 128) x all N outputs (UMMA N = n_tile <= 256),
// FP32 accumulators in tensor memory (n_tile columns).  K runs in chunks of
// 32 FP32 (one 128-byte swizzle row) through a two-stage TMA pipeline.
// Split-TF32: the line tile is split in shared memory into hi = tf32(x) and
// lo = tf32(x - hi); the matrix comes pre-split; three MMAs per K step
// (hi*hi + hi*lo + lo*hi) keep FP32-level accuracy.
//
// Warp roles (256 threads): warp 0 issues TMA loads, warp 1 owns tensor
// memory and issues the MMAs (one elected lane), warps 4..7 split the line
// tiles and then drain the accumulators (warp 4+q reads TMEM lanes 32q..).
// Every mbarrier wait is bounded (~1 s); a wait that gives up raises the
// CTA's abort flag and the device error word, and the CTA drains its copies
// and MMAs (bounded) and frees its tensor memory before returning.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "umma.h"

namespace cheb {

namespace {

constexpr int kBM = 128;     // lines per CTA
constexpr int kBK = 32;      // K per pipeline stage (128 bytes of FP32)
constexpr int kStages = 2;
constexpr int kUThreads = 256;
constexpr long long kWaitCycles = 1ll << 31;  // ~1 s at 2 GHz

__device__ int g_umma_err;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `parity` to complete.  Gives up (false) when the
// CTA's abort flag is raised or after kWaitCycles, raising the flag itself.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicOr(&g_umma_err, 1);
      return false;
    }
  }
  return true;
}
// Same, ignoring the abort flag (teardown drains).
__device__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > kWaitCycles) {
      atomicOr(&g_umma_err, 2);
      return false;
    }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row core-matrix groups 1024 bytes apart (SBO); LBO unused for this
// layout; descriptor version 1 (bits 46-47); swizzle mode 2 (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (load + wait in one
// block so no use of the registers is scheduled before the wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void __launch_bounds__(kUThreads, 1)
    umma_tf32x3_rot_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmWh,
                           const __grid_constant__ CUtensorMap tmWl, float* __restrict__ Y, int M, int N, int K,
                           int n_tile, int tmem_cols, const UmmaEpi ep) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t xbytes = kBM * 128u, wbytes = (uint32_t)n_tile * 128u;
  const uint32_t stage_bytes = 2u * xbytes + 2u * wbytes;  // [Xh | Xl | Wh | Wl]
  const uint32_t bars = base + kStages * stage_bytes;
  auto full = [&](int s) { return bars + 8u * s; };
  auto conv = [&](int s) { return bars + 8u * (kStages + s); };
  auto empty = [&](int s) { return bars + 8u * (2 * kStages + s); };
  const uint32_t done = bars + 8u * (3 * kStages);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + kStages * stage_bytes + 8 * (3 * kStages + 1));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int nchunks = (K + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(conv(s), 128);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmWh)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmWl)) : "memory");
      int last[kStages];
      for (int s = 0; s < kStages; ++s) last[s] = -1;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % kStages;
        const uint32_t ph = (uint32_t)(c / kStages) & 1u;
        if (!mbar_wait(empty(s), ph ^ 1u, abort_flag)) break;
        const uint32_t st = base + s * stage_bytes;
        mbar_expect_tx(full(s), xbytes + 2u * wbytes);
        tma_load_2d(st, &tmX, full(s), c * kBK, m0);
        tma_load_2d(st + 2u * xbytes, &tmWh, full(s), c * kBK, 0);
        tma_load_2d(st + 2u * xbytes + wbytes, &tmWl, full(s), c * kBK, 0);
        last[s] = c;
      }
      if (*abort_flag)  // drain copies still in flight before the CTA exits
        for (int s = 0; s < kStages; ++s)
          if (last[s] >= 0) mbar_drain(full(s), (uint32_t)(last[s] / kStages) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(kBM, n_tile);
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % kStages;
        const uint32_t ph = (uint32_t)(c / kStages) & 1u;
        if (!mbar_wait(conv(s), ph, abort_flag)) break;
        if (!mbar_wait(full(s), ph, abort_flag)) break;
        tc_fence_after();
        const uint32_t st = base + s * stage_bytes;
#pragma unroll
        for (int kk = 0; kk < kBK / 8; ++kk) {
          const uint64_t ah = sdesc_k_sw128(st + 32u * kk);
          const uint64_t al = sdesc_k_sw128(st + xbytes + 32u * kk);
          const uint64_t bh = sdesc_k_sw128(st + 2u * xbytes + 32u * kk);
          const uint64_t bl = sdesc_k_sw128(st + 2u * xbytes + wbytes + 32u * kk);
          umma_tf32(tmem, ah, bh, idesc, (c | kk) != 0);
          umma_tf32(tmem, ah, bl, idesc, 1u);
          umma_tf32(tmem, al, bh, idesc, 1u);
        }
        umma_commit(empty(s));
      }
      umma_commit(done);
      mbar_drain(done, 0);  // no MMA may be in flight when TMEM is freed
    }
    __syncwarp();
  } else if (warp >= 4) {
    const int t = threadIdx.x - 128;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c % kStages;
      const uint32_t ph = (uint32_t)(c / kStages) & 1u;
      if (!mbar_wait(full(s), ph, abort_flag)) {
        ok = false;
        break;
      }
      float4* xh = reinterpret_cast<float4*>(gbase + s * stage_bytes);
      float4* xl = reinterpret_cast<float4*>(gbase + s * stage_bytes + xbytes);
#pragma unroll 4
      for (int i = t; i < (int)(xbytes / 16); i += 128) {
        const float4 v = xh[i];
        float4 h, l;
        h.x = tf32_rna(v.x); l.x = tf32_rna(v.x - h.x);
        h.y = tf32_rna(v.y); l.y = tf32_rna(v.y - h.y);
        h.z = tf32_rna(v.z); l.z = tf32_rna(v.z - h.z);
        h.w = tf32_rna(v.w); l.w = tf32_rna(v.w - h.w);
        xh[i] = h;
        xl[i] = l;
      }
      // make the generic-proxy writes visible to the tensor cores
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(conv(s));
    }
    if (ok) ok = mbar_wait(done, 0, abort_flag);
    tc_fence_after();
    if (ok) {
      const int q = warp & 3;
      const int row = m0 + 32 * q + lane;
      const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
      int rf = row, rs = 0;
      bool rv = row < M;
      if (ep.mode != 0) {
        rs = row / ep.mpf;
        rf = row - rs * ep.mpf;
        rv = rv && rf < ep.mf && rs < ep.ms;
      }
      float lrow = 0.f;
      if (ep.mode == 1 && rv) lrow = ep.lf[rf] + (ep.ls ? ep.ls[rs] : 0.f);
      const long long xb = ep.xoff + rf * ep.xs_f + rs * ep.xs_s;
      float s0 = 0.f, sN = 0.f;
      for (int col = 0; col < n_tile; col += 16) {
        float v[16];
        tmem_ld16(tl + (uint32_t)col, v);
        if (ep.mode == 0) {
          if (row < M) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col + j < N) Y[(size_t)(col + j) * M + row] = v[j];
          }
        } else if (ep.mode == 1) {
          if (row < M) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = col + j;
              if (n < N) {
                const float fac = (rv && n < ep.mc) ? 1.f / (ep.kref * (lrow + ep.lc[n])) : 0.f;
                Y[(size_t)n * M + row] = v[j] * fac;
              }
            }
          }
        } else if (rv) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = col + j;
            if (n < ep.mc) {
              ep.x[xb + n * ep.xs_c] = v[j];
              s0 += ep.G[n] * v[j];
              sN += ep.G[ep.mc + n] * v[j];
            }
          }
        }
      }
      if (ep.mode == 2 && rv) {
        const long long p0 = xb - ep.xs_c, pN = p0 + (long long)(ep.ncol - 1) * ep.xs_c;
        const float r0 = ep.r[p0], rN = ep.r[pN];
        ep.x[p0] = s0 + ep.Binv[0] * r0 + ep.Binv[1] * rN;
        ep.x[pN] = sN + ep.Binv[2] * r0 + ep.Binv[3] * rN;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D FP32 tensor map: `rows` rows of `inner` contiguous floats, box of
// 32 floats (one 128-byte swizzle row) x box_rows rows.
int make_map(CUtensorMap* m, const float* ptr, int inner, int rows, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return CHEB_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed");
    return CHEB_ERR_CUDA;
  }
  return CHEB_OK;
}

size_t smem_bytes(int n_tile) {
  return (size_t)kStages * (2u * kBM * 128u + 2u * (size_t)n_tile * 128u) + 1024 + 8 * (3 * kStages + 1) + 8;
}

}  // namespace

int umma_n_tile(int N) { return (N + 15) / 16 * 16; }

bool umma_ok(int M, int N, int K) {
  return M >= kBM && N >= 32 && N <= 256 && K >= 32 && K % 4 == 0;
}

void tf32_split_host(const double* x, size_t n, float* hi, float* lo) {
  // round to nearest, ties away from zero, keeping 10 explicit mantissa bits
  auto rna = [](float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
  };
  for (size_t i = 0; i < n; ++i) {
    const float f = (float)x[i];
    hi[i] = rna(f);
    lo[i] = rna((float)(x[i] - (double)hi[i]));
  }
}

int umma_tf32x3_rot(const float* X, const float* Wh, const float* Wl, float* Y, int M, int N, int K,
                    const UmmaEpi& ep, cudaStream_t s) {
  if (!umma_ok(M, N, K) || (((uintptr_t)X | (uintptr_t)Wh | (uintptr_t)Wl) & 15)) {
    set_error("umma_tf32x3_rot: unsupported shape or alignment");
    return CHEB_ERR_UNSUPPORTED;
  }
  const int n_tile = umma_n_tile(N);
  int tmem_cols = 32;
  while (tmem_cols < n_tile) tmem_cols *= 2;
  CUtensorMap mx, mh, ml;
  int st;
  if ((st = make_map(&mx, X, K, M, kBM))) return st;
  if ((st = make_map(&mh, Wh, K, n_tile, n_tile))) return st;
  if ((st = make_map(&ml, Wl, K, n_tile, n_tile))) return st;
  const size_t sm = smem_bytes(n_tile);
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(umma_tf32x3_rot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_bytes(256));
  });
  CHEB_CUDA(attr_err);
  const int grid = (M + kBM - 1) / kBM;
  umma_tf32x3_rot_kernel<<<grid, kUThreads, sm, s>>>(mx, mh, ml, Y, M, N, K, n_tile, tmem_cols, ep);
  CHEB_LAUNCH_CHECK("umma_tf32x3_rot_kernel");
  return CHEB_OK;
}

int umma_take_error() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_umma_err, sizeof(int)) != cudaSuccess) return -1;
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_umma_err, &zero, sizeof(int));
  }
  return v;
}

}  // namespace cheb
