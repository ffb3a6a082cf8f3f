// Tensor-product contraction on the 5th-generation tensor cores (tcgen05).
//
// The fast-diagonalization preconditioner applies S^{-1} and S along each
// axis of the compact interior array: a dense (m_a x m_a) matrix against
// every a-line.  Contracting along the contiguous axis and writing the
// result transposed ([n][rows]) rotates the axes (x,y,z) -> (y,z,x), so three
// consecutive contractions return to the original layout and every operand
// is K-major: X rows (lines) as the MMA A operand, the matrix rows as B.
//
// Tile: 128 lines (UMMA M = 128) x all N outputs (UMMA N = n_tile <= 256),
// FP32 accumulators in tensor memory.  The kernel is persistent (one CTA per
// SM, tiles strided by the grid) with two accumulators, so the epilogue of
// one tile overlaps the MMAs of the next.  K runs in chunks of BK FP32
// (BK = 16: 64-byte swizzle, 4 stages; BK = 32: 128-byte swizzle, 2 stages)
// through a TMA ring that continues across tiles.  Split-TF32: the line tile
// is split in shared memory into hi = tf32(x) and lo = tf32(x - hi); the
// matrix comes pre-split; three MMAs per K step (hi*hi + hi*lo + lo*hi) keep
// FP32-level accuracy.
//
// Warp roles (384 threads): warp 0 issues TMA loads, warp 1 owns tensor
// memory and issues the MMAs (one lane), warps 4..7 split the line tiles,
// warps 8..11 drain the accumulators (warp 8+q reads TMEM lanes 32q..).
// Every mbarrier wait is bounded (~1 s); a wait that gives up raises the
// CTA's abort flag and the device error word, and the CTA drains its copies
// and MMAs (bounded) and frees its tensor memory before returning.
#include <cuda.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "umma.h"

namespace cheb {

namespace {

constexpr int kBM = 128;  // lines per tile
constexpr int kUThreads = 384;
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
// One bounded probe of the phase: the thread may sleep in hardware up to
// kSuspendNs until the phase completes (so waiting warps do not take issue
// slots from the working ones).
constexpr uint32_t kSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendNs)
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

// Shared-memory matrix descriptor of a K-major operand whose rows are
// BK * 4 bytes (the swizzle span): 128-byte swizzle (mode 2) for BK = 32,
// 64-byte swizzle (mode 4) for BK = 16; 8-row core-matrix groups 8 * BK * 4
// bytes apart (SBO); LBO unused for swizzled K-major layouts; descriptor
// version 1 (bits 46-47).  Advancing the start address by 32 bytes selects
// the next K = 8 step inside the swizzle row.
template <int BK>
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * BK * 4) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(BK == 32 ? 2 : 4) << 61;
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

// Two x16 loads (32 columns) behind one wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31},"
      " [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr), "r"(taddr + 16u)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Hardware reciprocal approximation (rcp.approx.ftz.f32, about 1 ulp): the
// eigenvalue division of the preconditioner needs FP32-level, not
// correctly rounded, accuracy.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int BK>
struct UmmaCfg {
  static constexpr int kStages = BK == 32 ? 2 : 4;
  static constexpr uint32_t kRow = BK * 4;  // bytes per operand row
};

template <int BK>
__global__ void __launch_bounds__(kUThreads, 1)
    umma_tf32x3_rot_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmWh,
                           const __grid_constant__ CUtensorMap tmWl, float* __restrict__ Y, int M, int N, int K,
                           int n_tile, int tmem_cols, const UmmaEpi ep) {
  constexpr int S = UmmaCfg<BK>::kStages;
  constexpr uint32_t RB = UmmaCfg<BK>::kRow;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t xbytes = kBM * RB, wbytes = (uint32_t)n_tile * RB;
  const uint32_t stage_bytes = 2u * xbytes + 2u * wbytes;  // [Xh | Xl | Wh | Wl]
  const uint32_t bars = base + S * stage_bytes;
  // barriers: full[S] conv[S] empty[S] tfull[2] tempty[2] fin
  auto full = [&](int s) { return bars + 8u * s; };
  auto conv = [&](int s) { return bars + 8u * (S + s); };
  auto empty = [&](int s) { return bars + 8u * (2 * S + s); };
  auto tfull = [&](int b) { return bars + 8u * (3 * S + b); };
  auto tempty = [&](int b) { return bars + 8u * (3 * S + 2 + b); };
  const uint32_t fin = bars + 8u * (3 * S + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + S * stage_bytes + 8 * (3 * S + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // per-column epilogue tables (eigenvalues of the column axis, or the two
  // rows of its elimination map G), staged once: global loads of them
  // could not be moved past the output stores
  float* tab = reinterpret_cast<float*>(gbase + S * stage_bytes + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (K + BK - 1) / BK;
  const int ntiles = (M + kBM - 1) / kBM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(conv(s), 128);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), 128);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (ep.mode == 1)
    for (int i = threadIdx.x; i < ep.mc; i += blockDim.x) tab[i] = ep.lc[i];
  else if (ep.mode == 2)
    for (int i = threadIdx.x; i < 2 * ep.mc; i += blockDim.x) tab[i] = ep.G[i];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmWh)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmWl)) : "memory");
      int last[S];
      for (int s = 0; s < S; ++s) last[s] = -1;
      int g = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int s = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(empty(s), ph ^ 1u, abort_flag)) break;
          const uint32_t st = base + s * stage_bytes;
          mbar_expect_tx(full(s), xbytes + 2u * wbytes);
          tma_load_2d(st, &tmX, full(s), c * BK, tile * kBM);
          tma_load_2d(st + 2u * xbytes, &tmWh, full(s), c * BK, 0);
          tma_load_2d(st + 2u * xbytes + wbytes, &tmWl, full(s), c * BK, 0);
          last[s] = g;
        }
      }
      if (*abort_flag)  // drain copies still in flight before the CTA exits
        for (int s = 0; s < S; ++s)
          if (last[s] >= 0) mbar_drain(full(s), (uint32_t)(last[s] / S) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(kBM, n_tile);
      int g = 0, it = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++it) {
        const int b = it & 1;
        const uint32_t d = tmem + (uint32_t)(b * tmem_cols);
        if (!mbar_wait(tempty(b), ((uint32_t)(it >> 1) & 1u) ^ 1u, abort_flag)) break;
        tc_fence_after();
        bool ok = true;
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int s = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(conv(s), ph, abort_flag) || !mbar_wait(full(s), ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + s * stage_bytes;
#pragma unroll
          for (int kk = 0; kk < BK / 8; ++kk) {
            const uint64_t ah = sdesc_k<BK>(st + 32u * kk);
            const uint64_t al = sdesc_k<BK>(st + xbytes + 32u * kk);
            const uint64_t bh = sdesc_k<BK>(st + 2u * xbytes + 32u * kk);
            const uint64_t bl = sdesc_k<BK>(st + 2u * xbytes + wbytes + 32u * kk);
            umma_tf32(d, ah, bh, idesc, (c | kk) != 0);
            umma_tf32(d, ah, bl, idesc, 1u);
            umma_tf32(d, al, bh, idesc, 1u);
          }
          umma_commit(empty(s));
        }
        if (!ok) break;
        umma_commit(tfull(b));
      }
      umma_commit(fin);
      mbar_drain(fin, 0);  // no MMA may be in flight when TMEM is freed
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    const int t = threadIdx.x - 128;
    int g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int c = 0; c < nchunks; ++c, ++g) {
        const int s = g % S;
        const uint32_t ph = (uint32_t)(g / S) & 1u;
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
    }
  } else if (warp >= 8) {
    const int q = warp & 3;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int b = it & 1;
      if (!mbar_wait(tfull(b), (uint32_t)(it >> 1) & 1u, abort_flag)) break;
      tc_fence_after();
      const int row = tile * kBM + 32 * q + lane;
      const uint32_t tl = tmem + (uint32_t)(b * tmem_cols) + ((uint32_t)(32 * q) << 16);
      int rf = row, rs = 0;
      bool rv = row < M;
      if (ep.mode != 0) {
        rs = row / ep.mpf;
        rf = row - rs * ep.mpf;
        rv = rv && rf < ep.mf && rs < ep.ms;
      }
      float lrow = 0.f;
      if (ep.mode == 1 && rv) lrow = ep.lf[rf] + (ep.ls ? ep.ls[rs] : 0.f);
      // full grids have < 2^31 points: 32-bit offsets
      const int xb = (int)ep.xoff + rf * (int)ep.xs_f + rs * (int)ep.xs_s;
      const int xc = (int)ep.xs_c;
      float s0 = 0.f, sN = 0.f;
      float* yrow = Y + row;
      for (int col = 0; col < n_tile; col += 32) {
        float v[32];
        if (col + 16 < n_tile) {
          tmem_ld32(tl + (uint32_t)col, v);
        } else {
          float h[16];
          tmem_ld16(tl + (uint32_t)col, h);
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = h[j];
#pragma unroll
          for (int j = 16; j < 32; ++j) v[j] = 0.f;
        }
        if (ep.mode == 0) {
          if (row < M) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (col + j < N) yrow[(size_t)(col + j) * M] = v[j];
          }
        } else if (ep.mode == 1) {
          // factors first (shared-memory reads batched ahead of the stores)
          float fac[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = col + j;
            fac[j] = (rv && n < ep.mc) ? rcp_approx(ep.kref * (lrow + tab[n])) : 0.f;
          }
          if (row < M) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (col + j < N) yrow[(size_t)(col + j) * M] = v[j] * fac[j];
          }
        } else if (rv) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = col + j;
            if (n < ep.mc) {
              s0 += tab[n] * v[j];
              sN += tab[ep.mc + n] * v[j];
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col + j < ep.mc) ep.x[xb + (col + j) * xc] = v[j];
        }
      }
      // accumulator drained: hand it back to the MMA issuer
      tc_fence_before();
      mbar_arrive(tempty(b));
      if (ep.mode == 2 && rv) {
        const int p0 = xb - xc, pN = p0 + (ep.ncol - 1) * xc;
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * tmem_cols)
                 : "memory");
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
// bk floats (one swizzle row: 128 bytes for bk = 32, 64 for bk = 16) x
// box_rows rows.
int make_map(CUtensorMap* m, const float* ptr, int inner, int rows, int box_rows, int bk) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return CHEB_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed");
    return CHEB_ERR_CUDA;
  }
  return CHEB_OK;
}

template <int BK>
size_t smem_bytes(int n_tile) {
  constexpr int S = UmmaCfg<BK>::kStages;
  // stages, alignment slack, barriers + TMEM slot + abort flag (256 B), tables (2 x 256 floats)
  return (size_t)S * (2u * kBM + 2u * (size_t)n_tile) * UmmaCfg<BK>::kRow + 1024 + 256 + 2048;
}

int sm_count() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 148;
  });
  return n;
}

// K chunk of the pipeline: 16 unless overridden by CHEB_UMMA_BK=32.
int chunk_k() {
  static int bk = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* e = std::getenv("CHEB_UMMA_BK");
    bk = (e && std::atoi(e) == 32) ? 32 : 16;
  });
  return bk;
}

template <int BK>
int launch_rot(const float* X, const float* Wh, const float* Wl, float* Y, int M, int N, int K, int n_tile,
               int tmem_cols, const UmmaEpi& ep, cudaStream_t s) {
  CUtensorMap mx, mh, ml;
  int st;
  if ((st = make_map(&mx, X, K, M, kBM, BK))) return st;
  if ((st = make_map(&mh, Wh, K, n_tile, n_tile, BK))) return st;
  if ((st = make_map(&ml, Wl, K, n_tile, n_tile, BK))) return st;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(umma_tf32x3_rot_kernel<BK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_bytes<BK>(256));
  });
  CHEB_CUDA(attr_err);
  const int ntiles = (M + kBM - 1) / kBM;
  const int grid = std::min(ntiles, sm_count());
  umma_tf32x3_rot_kernel<BK><<<grid, kUThreads, smem_bytes<BK>(n_tile), s>>>(mx, mh, ml, Y, M, N, K, n_tile,
                                                                               tmem_cols, ep);
  CHEB_LAUNCH_CHECK("umma_tf32x3_rot_kernel");
  return CHEB_OK;
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
  return chunk_k() == 32 ? launch_rot<32>(X, Wh, Wl, Y, M, N, K, n_tile, tmem_cols, ep, s)
                         : launch_rot<16>(X, Wh, Wl, Y, M, N, K, n_tile, tmem_cols, ep, s);
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
