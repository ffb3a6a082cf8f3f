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
// (BK = 16: 64-byte swizzle; BK = 32: 128-byte swizzle) through a TMA ring
// that continues across tiles.  Split-TF32: the line tile is split in shared
// memory into hi = tf32(x) and lo = tf32(x - hi); the matrix comes pre-split,
// three MMAs per K step (hi*hi + hi*lo + lo*hi) keep FP32-level accuracy
// (BK = 16, 4 stages); or the matrix is taken as exactly TF32 and two MMAs
// (hi*W + lo*W) apply it to FP32 accuracy (BK = 32, 3 stages).
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
#include <vector>
#include <cstring>
#include <mutex>

#include "device.cuh"
#include "hostmath.h"
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
// CTA's abort flag is raised or after `limit` cycles (kWaitCycles in the
// kernels), raising the flag and the device error word itself.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                          long long limit = kWaitCycles) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
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

// Self-test of the bounded waits and the abort path: the CTA allocates
// tensor memory as the contraction kernels do, thread 0 waits (with a short
// limit) on a freshly initialised mbarrier that nothing ever arrives on, the
// wait gives up and raises the abort flag and the device error word, and the
// CTA frees its tensor memory and returns.  No copy or MMA is ever issued, so
// nothing is in flight when the CTA ends.
__global__ void __launch_bounds__(64, 1) wait_selftest_kernel(long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0u, &abort_flag, limit);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(&tmem_slot);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
  }
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

// Stage ring of the contraction: [Xh | Xl | Wh | Wl] per stage for three
// products, [Xh | Xl | Wh] for two, as many stages as about 192 KB hold (the
// line tile is the one operand streamed from HBM: more stages keep more of
// it in flight).
template <int BK, int TERMS>
struct UmmaCfg {
  static constexpr int kStages = TERMS == 3 ? (BK == 32 ? 2 : 4) : (BK == 32 ? 3 : 6);
  static constexpr uint32_t kRow = BK * 4;  // bytes per operand row
};

// TERMS = 3: W given as its split pair, three products per K step.
// TERMS = 2: W is exactly TF32 (Wl = 0 and never loaded), two products
// Xh W + Xl W per K step: the matrix is applied as given, the line tile
// still to FP32 accuracy.
template <int BK, int TERMS>
__global__ void __launch_bounds__(kUThreads, 1)
    umma_tf32x3_rot_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmWh,
                           const __grid_constant__ CUtensorMap tmWl, float* __restrict__ Y, int M, int N, int K,
                           int n_tile, int tmem_cols, const UmmaEpi ep) {
  // a converged instance of a batched solve: nothing is initialised or
  // allocated yet, every thread of the CTA returns
  if (ep.active && *ep.active == 0) return;
  constexpr int S = UmmaCfg<BK, TERMS>::kStages;
  constexpr uint32_t RB = UmmaCfg<BK, TERMS>::kRow;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t xbytes = kBM * RB, wbytes = (uint32_t)n_tile * RB;
  const uint32_t stage_bytes = 2u * xbytes + (uint32_t)(TERMS - 1) * wbytes;  // [Xh | Xl | Wh (| Wl)]
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
      if (TERMS == 3) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmWl)) : "memory");
      int last[S];
      for (int s = 0; s < S; ++s) last[s] = -1;
      int g = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int s = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(empty(s), ph ^ 1u, abort_flag)) break;
          const uint32_t st = base + s * stage_bytes;
          mbar_expect_tx(full(s), xbytes + (uint32_t)(TERMS - 1) * wbytes);
          tma_load_2d(st, &tmX, full(s), c * BK, tile * kBM);
          tma_load_2d(st + 2u * xbytes, &tmWh, full(s), c * BK, 0);
          if (TERMS == 3) tma_load_2d(st + 2u * xbytes + wbytes, &tmWl, full(s), c * BK, 0);
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
            umma_tf32(d, ah, bh, idesc, (c | kk) != 0);
            if (TERMS == 3) umma_tf32(d, ah, sdesc_k<BK>(st + 2u * xbytes + wbytes + 32u * kk), idesc, 1u);
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

template <int BK, int TERMS>
size_t smem_bytes(int n_tile) {
  constexpr int S = UmmaCfg<BK, TERMS>::kStages;
  // stages, alignment slack, barriers + TMEM slot + abort flag (256 B), tables (2 x 256 floats)
  return (size_t)S * (2u * kBM + (TERMS - 1u) * (size_t)n_tile) * UmmaCfg<BK, TERMS>::kRow + 1024 + 256 + 2048;
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

// K chunk of the contraction's ring: 16 columns (64-byte swizzle) for the
// three-product form, 32 (128-byte swizzle) for the two-product form, where
// the freed matrix slots leave room for three 64 KB stages (measured at 257^3:
// 0.433 ms per preconditioner application against 0.455 ms with 16); the
// environment variable CHEB_UMMA_BK = 16 or 32 overrides both.
int chunk_k(bool three_products) {
  static int forced = -1;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* e = std::getenv("CHEB_UMMA_BK");
    const int v = e ? std::atoi(e) : 0;
    forced = (v == 16 || v == 32) ? v : 0;
  });
  if (forced) return forced;
  return three_products ? 16 : 32;
}

template <int BK>
int launch_rot(const float* X, const float* Wh, const float* Wl, float* Y, int M, int N, int K, int n_tile,
               int tmem_cols, const UmmaEpi& ep, cudaStream_t s) {
  CUtensorMap mx, mh, ml;
  int st;
  if ((st = make_map(&mx, X, K, M, kBM, BK))) return st;
  if ((st = make_map(&mh, Wh, K, n_tile, n_tile, BK))) return st;
  // two-product form: the map of Wl is passed but never read
  if ((st = make_map(&ml, Wl ? Wl : Wh, K, n_tile, n_tile, BK))) return st;
  const int ntiles = (M + kBM - 1) / kBM;
  const int grid = std::min(ntiles, sm_count());
  if (Wl) {
    if ((st = ensure_smem_attr((const void*)umma_tf32x3_rot_kernel<BK, 3>, smem_bytes<BK, 3>(256)))) return st;
    umma_tf32x3_rot_kernel<BK, 3><<<grid, kUThreads, smem_bytes<BK, 3>(n_tile), s>>>(mx, mh, ml, Y, M, N, K, n_tile,
                                                                                  tmem_cols, ep);
  } else {
    if ((st = ensure_smem_attr((const void*)umma_tf32x3_rot_kernel<BK, 2>, smem_bytes<BK, 2>(256)))) return st;
    umma_tf32x3_rot_kernel<BK, 2><<<grid, kUThreads, smem_bytes<BK, 2>(n_tile), s>>>(mx, mh, ml, Y, M, N, K, n_tile,
                                                                                  tmem_cols, ep);
  }
  CHEB_LAUNCH_CHECK("umma_tf32x3_rot_kernel");
  return CHEB_OK;
}


// ---------------------------------------------------------------------------
// Tensor-core route of the operator apply.  The line derivative is the dense
// collocation matrix, f' = D f on every line (Sec. 2.2), so the interior rows
// of A u = -sum_a D_a (K (D_a u)) are two contractions per axis:
//   phase 1: Q = K * (D_a u) on every node, and (D_a u) at the two ends of
//            every a-line (the normal derivatives of the Neumann rows);
//   phase 2: out (+)= -(D_a Q) on interior nodes, and the boundary rows
//            (Dirichlet: u; Neumann of this axis: the signed end derivative)
//            with the owner rule of the line passes.
// Tile: 128 a-lines (UMMA M = 128) x nA output points (UMMA N, in groups of
// at most 256 columns), K = the points of the line in chunks of 16 (64-byte
// swizzle).  The converter warps read the line tile from global memory (the
// odd grid extents rule out TMA for it: rows of 257 floats are not 16-byte
// strided) and write its TF32 hi/lo split in the swizzled K-major layout;
// D comes pre-split by TMA.  Same warp roles, bounded waits and teardown as
// the contraction kernel above.
// ---------------------------------------------------------------------------
constexpr int kDK = 16;      // K chunk (one 64-byte swizzle row)
constexpr int kDStages = 3;  // D / split-tile stages
constexpr int kRaw = 3;      // raw line-tile slots filled by cp.async (two chunks ahead)
constexpr int kRawFloats = 128 * 17;  // one slot: 128 lines x 16 points (x-lines: rows padded to 17)

// Line L of axis a starts at base(L) with point stride stride(); 32-bit
// offsets (grids have < 2^31 points).
struct LineGeo {
  int axis, nx, ny, n, nl;
  __device__ __forceinline__ int base(int L) const {
    return axis == 0 ? L * nx : (axis == 1 ? (L / nx) * (nx * ny) + (L % nx) : L);
  }
  __device__ __forceinline__ int stride() const { return axis == 0 ? 1 : (axis == 1 ? nx : nx * ny); }
  __device__ __forceinline__ void node(int L, int pt, int& i, int& j, int& k) const {
    if (axis == 0) { i = pt; j = L % ny; k = L / ny; }
    else if (axis == 1) { i = L % nx; j = pt; k = L / nx; }
    else { i = L % nx; j = L / nx; k = pt; }
  }
};

struct DenseArgs {
  Geom g;
  int phase, first;
  const float* src;  // u (phase 1) or Q (phase 2)
  const float* K;    // phase 1
  float* Q;          // phase 1 output
  float2* ends;      // (D u) at points 0 and n-1 of every line
  const float* u;    // phase 2: Dirichlet rows
  float* out;        // phase 2
  const float* Dend; // phase 1, 257-point lines: row n-1 of D (FP32); that output point
                     // is a dot product in the converters, so the MMA needs N = 256 only
};

// shared-memory bytes of the dense pass for nA D rows per stage: alignment
// slack, stages, barriers, raw line-tile slots, epilogue prefetch (8 warps x
// 3 slots x 512 floats), row n-1 of D, the converters' end values, x-line
// class tables (8 warps x 128)
size_t dense_smem_bytes(int nA) {
  return 1024 + (size_t)kDStages * (2u * kBM + 2u * (size_t)nA) * (kDK * 4) + 256 + kRaw * kRawFloats * 4 +
         8 * 1536 * 4 + 272 * 4 + 2 * 128 * 4 + 8 * 128 * 4;
}

__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc, bool valid) {
  // 4-byte asynchronous copy; an invalid element (gsrc still a valid address)
  // copies zero source bytes and fills zero
  const uint32_t sa = smem_u32(sdst);
  const uint32_t n = valid ? 4u : 0u;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NW>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NW) : "memory"); }

// Boundary rows in phase 2.  A line either runs through the interior of the
// other axes (its points 1 .. n-2 are interior nodes: out (+)= -C), or lies in
// a face of another axis (its points 1 .. n-2 all have the same owner face:
// Dirichlet -> u on the first pass, Neumann of the other axis -> 0 on the
// first pass, else untouched).  The two line ends are boundary nodes of this
// axis and take the owner rule per node.  The grid and boundary set are held
// in registers (a Dirichlet-face bit mask).
struct BcInfo {
  int nx, ny, nz, dim, dmask, first, axis;
  __device__ __forceinline__ int owner(int i, int j, int k) const {
    // Dirichlet faces beat Neumann faces, then the lowest axis (node index 0
    // of an axis is its hi face 2a + 1, index n - 1 the lo face 2a)
    int fd = -1, fn = -1;
    const int f0 = i == 0 ? 1 : (i == nx - 1 ? 0 : -1);
    const int f1 = dim > 1 ? (j == 0 ? 3 : (j == ny - 1 ? 2 : -1)) : -1;
    const int f2 = dim > 2 ? (k == 0 ? 5 : (k == nz - 1 ? 4 : -1)) : -1;
    if (f2 >= 0) { if ((dmask >> f2) & 1) fd = f2; else fn = f2; }
    if (f1 >= 0) { if ((dmask >> f1) & 1) fd = f1; else fn = f1; }
    if (f0 >= 0) { if ((dmask >> f0) & 1) fd = f0; else fn = f0; }
    return fd >= 0 ? fd : fn;
  }
};
// class of the points 1 .. n-2 of a line (phase 2)
enum LineClass { kLineInterior = 0, kLineCopyU = 1, kLineZero = 2, kLineSkip = 3 };

// threads of the dense pass: 8 warps of producer / MMA / converters plus 8
// epilogue warps (two per TMEM lane quarter)
template <bool XAX>
__host__ __device__ constexpr int dense_epi_warps() { return 8; }
template <bool XAX>
__host__ __device__ constexpr int dense_threads() { return 256 + 32 * dense_epi_warps<XAX>(); }
// D rows held per stage: x-lines use whole 128-row M tiles
template <bool XAX>
__host__ __device__ constexpr int dense_rows(int nA) { return XAX ? (nA + 127) / 128 * 128 : nA; }

template <bool XAX>
__global__ void __launch_bounds__(dense_threads<XAX>(), 1)
    dense_pass_kernel(const __grid_constant__ CUtensorMap tmDh, const __grid_constant__ CUtensorMap tmDl,
                      const LineGeo lg, const DenseArgs A, int nA, int tmem_cols, int nbuf) {
  constexpr int S = kDStages;
  constexpr uint32_t RB = kDK * 4;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  // x-lines swap the MMA roles (A = D: points on the TMEM lanes, B = the line
  // tile), so D occupies whole 128-row M tiles
  const int nAx = dense_rows<XAX>(nA);
  const uint32_t xbytes = kBM * RB, dbytes = (uint32_t)nAx * RB;
  const uint32_t stage_bytes = 2u * xbytes + 2u * dbytes;  // [Xh | Xl | Dh | Dl]
  const uint32_t bars = base + S * stage_bytes;
  auto full = [&](int s) { return bars + 8u * s; };
  auto conv = [&](int s) { return bars + 8u * (S + s); };
  auto empty = [&](int s) { return bars + 8u * (2 * S + s); };
  auto tfull = [&](int b) { return bars + 8u * (3 * S + b); };
  auto tempty = [&](int b) { return bars + 8u * (3 * S + 2 + b); };
  const uint32_t fin = bars + 8u * (3 * S + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + S * stage_bytes + 8 * (3 * S + 7));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* rawt = reinterpret_cast<float*>(gbase + S * stage_bytes + 256);  // kRaw slots of the line tile
  float* stg = rawt + kRaw * kRawFloats;                                   // epilogue prefetch: 8 x 1536
  float* dend = stg + 8 * 1536;                                            // 272: row n-1 of D
  float* gend = dend + 272;                                                // 2 x 128 end values
  int* clsw = reinterpret_cast<int*>(gend + 256);                          // x-lines: 8 x 128 line classes
  const bool xend = A.phase == 1 && A.Dend != nullptr;
  // end-value barriers (converters -> epilogue), one per accumulator buffer
  auto endb = [&](int b) { return bars + 8u * (3 * S + 5) + 8u * b; };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = lg.n;
  const int nchunks = (n + kDK - 1) / kDK;
  const int ntiles = (lg.nl + kBM - 1) / kBM;
  const int ng = nA > 256 ? 2 : 1;  // MMA column groups

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(conv(s), 128);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), 32 * dense_epi_warps<XAX>());
      mbar_init(endb(b), 128);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (xend)
    for (int i = threadIdx.x; i < 272; i += blockDim.x) dend[i] = i < n ? A.Dend[i] : 0.f;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(nbuf * tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tmem_slot);

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmDh)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmDl)) : "memory");
      int last[S];
      for (int s = 0; s < S; ++s) last[s] = -1;
      int g = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int s = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(empty(s), ph ^ 1u, abort_flag)) break;
          const uint32_t st = base + s * stage_bytes + 2u * xbytes;
          mbar_expect_tx(full(s), 2u * dbytes);
          // D rows in two boxes of nAx / 2 rows each (a box has at most 256 rows)
          tma_load_2d(st, &tmDh, full(s), c * kDK, 0);
          tma_load_2d(st + dbytes / 2, &tmDh, full(s), c * kDK, nAx / 2);
          tma_load_2d(st + dbytes, &tmDl, full(s), c * kDK, 0);
          tma_load_2d(st + dbytes + dbytes / 2, &tmDl, full(s), c * kDK, nAx / 2);
          last[s] = g;
        }
      }
      if (*abort_flag)
        for (int s = 0; s < S; ++s)
          if (last[s] >= 0) mbar_drain(full(s), (uint32_t)(last[s] / S) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int g = 0, it = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++it) {
        const int b = it % nbuf, use = it / nbuf;
        const uint32_t d = tmem + (uint32_t)(b * tmem_cols);
        if (!mbar_wait(tempty(b), ((uint32_t)use & 1u) ^ 1u, abort_flag)) break;
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
          for (int kk = 0; kk < kDK / 8; ++kk) {
            if (XAX) {
              // A = D rows of M tile mt (points), B = the line tile (N = 128)
              const uint64_t bh = sdesc_k<kDK>(st + 32u * kk);
              const uint64_t bl = sdesc_k<kDK>(st + xbytes + 32u * kk);
              const uint32_t idesc = idesc_tf32(kBM, kBM);
              for (int mt = 0; mt < nAx / 128; ++mt) {
                const uint32_t aoff = (uint32_t)mt * 128u * RB;
                const uint64_t ah = sdesc_k<kDK>(st + 2u * xbytes + aoff + 32u * kk);
                const uint64_t al = sdesc_k<kDK>(st + 2u * xbytes + dbytes + aoff + 32u * kk);
                const uint32_t dc = d + (uint32_t)(mt * 128);
                umma_tf32(dc, ah, bh, idesc, (c | kk) != 0);
                umma_tf32(dc, ah, bl, idesc, 1u);
                umma_tf32(dc, al, bh, idesc, 1u);
              }
              continue;
            }
            const uint64_t ah = sdesc_k<kDK>(st + 32u * kk);
            const uint64_t al = sdesc_k<kDK>(st + xbytes + 32u * kk);
            for (int gi = 0; gi < ng; ++gi) {
              const int nb = gi == 0 ? (nA < 256 ? nA : 256) : nA - 256;
              const uint32_t idesc = idesc_tf32(kBM, nb);
              const uint32_t boff = (uint32_t)gi * 256u * RB;
              const uint64_t bh = sdesc_k<kDK>(st + 2u * xbytes + boff + 32u * kk);
              const uint64_t bl = sdesc_k<kDK>(st + 2u * xbytes + dbytes + boff + 32u * kk);
              const uint32_t dc = d + (uint32_t)(gi * 256);
              umma_tf32(dc, ah, bh, idesc, (c | kk) != 0);
              umma_tf32(dc, ah, bl, idesc, 1u);
              umma_tf32(dc, al, bh, idesc, 1u);
            }
          }
          umma_commit(empty(s));
        }
        if (!ok) break;
        umma_commit(tfull(b));
      }
      umma_commit(fin);
      mbar_drain(fin, 0);
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    // converters: one line per thread.  The line tile of chunk c + 2 is copied
    // by cp.async into a raw slot while chunk c is split, so the global loads
    // stay in flight across the per-chunk proxy fence.
    const int t = threadIdx.x - 128;
    const int stride = lg.stride();
    int g = 0, tile_it = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tile_it) {
      const int L0 = tile * kBM, L = L0 + t;
      const bool lv = L < lg.nl;
      const int lb = lv ? lg.base(L) : 0;
      // raw slot layout: x-lines [line][17] (16 threads per line, coalesced);
      // other axes [point][128] (a thread per line, coalesced across lines)
      auto issue = [&](int c) {
        float* slot = rawt + (c % kRaw) * kRawFloats;
#pragma unroll
        for (int r = 0; r < kDK; ++r) {
          if (XAX) {
            const int e = t + 128 * r, m = e >> 4, kk = e & 15, pt = c * kDK + kk, Lm = L0 + m;
            const bool v = Lm < lg.nl && pt < n;
            cp_async4(slot + m * 17 + kk, A.src + (v ? Lm * lg.nx + pt : 0), v);
          } else {
            const int pt = c * kDK + r;
            const bool v = lv && pt < n;
            cp_async4(slot + r * 128 + t, A.src + (v ? lb + pt * stride : 0), v);
          }
        }
        cp_async_commit();
      };
      issue(0);
      if (nchunks > 1) issue(1);
      float gacc = 0.f;  // row n-1 of D against this thread's line (xend)
      for (int c = 0; c < nchunks; ++c, ++g) {
        const int s = g % S;
        const uint32_t ph = (uint32_t)(g / S) & 1u;
        if (c + 2 < nchunks) {
          issue(c + 2);
          cp_async_wait<2>();
        } else if (c + 1 < nchunks) {
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        if (XAX) asm volatile("bar.sync 1, 128;" ::: "memory");  // rows filled by 16 threads each
        const float* slot = rawt + (c % kRaw) * kRawFloats;
        float v[kDK];
#pragma unroll
        for (int kk = 0; kk < kDK; ++kk) v[kk] = XAX ? slot[t * 17 + kk] : slot[kk * 128 + t];
        if (xend) {
#pragma unroll
          for (int kk = 0; kk < kDK; ++kk) gacc = fmaf(dend[c * kDK + kk], v[kk], gacc);
        }
        // the stage is free once the MMAs of its previous use completed
        if (!mbar_wait(empty(s), ph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        uint8_t* xh = gbase + s * stage_bytes + t * RB;
        uint8_t* xl = xh + xbytes;
#pragma unroll
        for (int q = 0; q < kDK / 4; ++q) {
          // 64-byte swizzle: 16-byte granule q of row t sits at q ^ ((t >> 1) & 3)
          const int gp = q ^ ((t >> 1) & 3);
          float4 h, l;
          h.x = tf32_rna(v[4 * q + 0]); l.x = tf32_rna(v[4 * q + 0] - h.x);
          h.y = tf32_rna(v[4 * q + 1]); l.y = tf32_rna(v[4 * q + 1] - h.y);
          h.z = tf32_rna(v[4 * q + 2]); l.z = tf32_rna(v[4 * q + 2] - h.z);
          h.w = tf32_rna(v[4 * q + 3]); l.w = tf32_rna(v[4 * q + 3] - h.w);
          *reinterpret_cast<float4*>(xh + gp * 16) = h;
          *reinterpret_cast<float4*>(xl + gp * 16) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (xend && c == nchunks - 1) {
          gend[(tile_it & 1) * 128 + t] = gacc;
          mbar_arrive(endb(tile_it & 1));
        }
        mbar_arrive(conv(s));
        // the raw slot of chunk c is refilled by issue(c + 3): all its readers
        // are past this point before any thread issues it (x-lines share rows)
        if (XAX) asm volatile("bar.sync 1, 128;" ::: "memory");
      }
      if (!ok) cp_async_wait<0>();  // no copy may land after the CTA gave up
    }
  } else if (warp >= 8) {
    BcInfo bi;
    bi.nx = A.g.n[0];
    bi.ny = A.g.n[1];
    bi.nz = A.g.n[2];
    bi.dim = A.g.dim;
    bi.dmask = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) bi.dmask |= (A.g.bc[f] == CHEB_DIRICHLET ? 1 : 0) << f;
    bi.first = A.first;
    bi.axis = lg.axis;
    const int phase = A.phase, first = A.first;
    const float* Kp = A.K;
    float* Qp = A.Q;
    float* outp = A.out;
    const float* up = A.u;
    // class of the points 1 .. n-2 of line L (phase 2), from its point 1
    auto line_class = [&](int L) {
      if (L >= lg.nl) return (int)kLineSkip;
      int ci, cj, ck;
      lg.node(L, 1, ci, cj, ck);
      const int o = bi.owner(ci, cj, ck);
      if (o < 0) return (int)kLineInterior;
      if (!first) return (int)kLineSkip;
      return ((bi.dmask >> o) & 1) ? (int)kLineCopyU : (int)kLineZero;
    };
    // the two ends of line L: boundary nodes of this axis, owner rule per node
    auto line_ends = [&](int L, int lb, int stride, float e0, float eN) {
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int pt = side ? n - 1 : 0;
        int i, jj, k;
        lg.node(L, pt, i, jj, k);
        const int idx = lb + pt * stride;
        const int o = bi.owner(i, jj, k);
        if ((bi.dmask >> o) & 1) {
          if (first) outp[idx] = up[idx];
        } else if ((o >> 1) == lg.axis) {
          // hi face (side 1) is line point 0, lo face (side 0) is point n - 1
          outp[idx] = (o & 1) ? e0 : -eN;
        } else if (first) {
          outp[idx] = 0.f;  // Neumann row of another axis: written by that axis' pass
        }
      }
    };
    if constexpr (XAX) {
      // x-lines: the accumulator holds points on the TMEM lanes and the
      // tile's 128 lines on the columns.  Warp 8 + 4 mt + q reads the points
      // mt * 128 + 32 q + lane of M tile mt, so for each line the 32 lanes
      // store 32 consecutive points (coalesced, no staging).  Global operands
      // of a 16-line chunk are prefetched by cp.async two chunks ahead; the
      // line classes of the tile sit in a per-warp table.
      const int mt = (warp - 8) >> 2, q = warp & 3;
      const int et = threadIdx.x - 256;  // epilogue thread, one per line in the tails
      const bool act = mt < nAx / 128;
      const int pt = mt * 128 + 32 * q + lane;
      const bool pin = pt > 0 && pt < n - 1;
      float* pf = stg + (warp - 8) * 1536;
      int* cw = clsw + (warp - 8) * 128;
      constexpr int PD = 2, NC = kBM / 16;
      int it = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int b = it % nbuf, use = it / nbuf;
        if (!mbar_wait(tfull(b), (uint32_t)use & 1u, abort_flag)) break;
        tc_fence_after();
        const int L0 = tile * kBM;
        if (phase == 2) {
#pragma unroll
          for (int r = 0; r < 4; ++r) cw[lane + 32 * r] = line_class(L0 + lane + 32 * r);
          __syncwarp();
        }
        const uint32_t tl = tmem + (uint32_t)(b * tmem_cols + mt * 128) + ((uint32_t)(32 * q) << 16);
        auto prefetch = [&](int c) {
          float* dst = pf + (c % (PD + 1)) * 512;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int Lr = L0 + 16 * c + j;
            bool v = act && Lr < lg.nl && pt < n;
            const float* src = Kp;
            if (phase == 2) {
              const int cl = cw[16 * c + j];
              v = v && pin && ((cl == kLineInterior && !first) || cl == kLineCopyU);
              src = cl == kLineCopyU ? up : outp;
            }
            cp_async4(dst + j * 32 + lane, (v ? src : Kp) + (v ? Lr * lg.nx + pt : 0), v);
          }
          cp_async_commit();
        };
        for (int c = 0; c < PD; ++c) prefetch(c);
        for (int c = 0; c < NC; ++c) {
          if (c + PD < NC) {
            prefetch(c + PD);
            cp_async_wait<PD>();
          } else if (NC - 1 - c >= 1) {
            cp_async_wait<1>();
          } else {
            cp_async_wait<0>();
          }
          const float* cur = pf + (c % (PD + 1)) * 512;
          float v[16];
          if (act) {
            tmem_ld16(tl + (uint32_t)(16 * c), v);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0.f;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int Lr = L0 + 16 * c + j;
            if (!act || Lr >= lg.nl || pt >= n) continue;
            const int idx = Lr * lg.nx + pt;
            const float ld = cur[j * 32 + lane];
            if (phase == 1) {
              __stcg(Qp + idx, ld * v[j]);
              float* ef = reinterpret_cast<float*>(A.ends + Lr);
              if (pt == 0) ef[0] = v[j];
              if (!xend && pt == n - 1) ef[1] = v[j];
            } else if (pin) {
              const int cl = cw[16 * c + j];
              if (cl == kLineInterior) __stcg(outp + idx, ld - v[j]);
              else if (cl == kLineCopyU) __stcg(outp + idx, ld);
              else if (cl == kLineZero) __stcg(outp + idx, 0.f);
            }
          }
        }
        // accumulator drained: hand it back to the MMA issuer
        tc_fence_before();
        mbar_arrive(tempty(b));
        // per-line tails, one epilogue thread per line of the tile
        if (et < 128) {
          const int L = L0 + et;
          if (xend) {
            // point n-1 of 257-point lines: the converters' dot product
            if (!mbar_wait(endb(b), (uint32_t)use & 1u, abort_flag)) break;
            if (L < lg.nl) {
              const float g = gend[b * 128 + et];
              const int idx = L * lg.nx + n - 1;
              Qp[idx] = Kp[idx] * g;
              reinterpret_cast<float*>(A.ends + L)[1] = g;
            }
          }
          if (phase == 2 && L < lg.nl) {
            const float2 e = A.ends[L];
            line_ends(L, L * lg.nx, 1, e.x, e.y);
          }
        }
        // the class table is rewritten next tile: this warp's readers are done
        __syncwarp();
      }
    } else {
      // strided lines: a thread per line (lanes along consecutive lines);
      // two epilogue groups share each TMEM lane quarter and take alternate
      // 16-column blocks; group 0 also writes the line-end rows
      const int q = warp & 3;
      const int grp = (warp - 8) >> 2;
      const int ngrp = dense_epi_warps<XAX>() / 4;
      const int stride = lg.stride();
      int it = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int b = it % nbuf, use = it / nbuf;
        if (!mbar_wait(tfull(b), (uint32_t)use & 1u, abort_flag)) break;
        tc_fence_after();
        const int L = tile * kBM + 32 * q + lane;
        const bool lv = L < lg.nl;
        const int lb = lv ? lg.base(L) : 0;
        const uint32_t tl = tmem + (uint32_t)(b * tmem_cols) + ((uint32_t)(32 * q) << 16);
        const int cls = phase == 2 ? line_class(L) : (int)kLineSkip;
        float e0 = 0.f, eN = 0.f;
        if (phase == 2 && lv) {
          const float2 e = A.ends[L];
          e0 = e.x;
          eN = e.y;
        }
        float gl = 0.f;  // D u at point n-1 (xend)
        if (xend) {
          if (!mbar_wait(endb(b), (uint32_t)use & 1u, abort_flag)) break;
          gl = gend[b * 128 + 32 * q + lane];
        }
        const int ncol = phase == 1 ? (xend ? n : nA) : n;
        // The global operands of the epilogue (K in phase 1; the accumulated
        // output or u in phase 2) are copied by cp.async two of this warp's
        // blocks ahead into 3 slots of 16 points x 32 lines (over the staging
        // area the x-lines use); each thread reads back only its own copies.
        float* pf = stg + (warp - 8) * 1536;
        constexpr int PD = 2, PS = 512, bw = 16;
        const int nblk = (ncol + bw - 1) / bw;
        const int nmy = (nblk - grp + ngrp - 1) / ngrp;  // this warp's blocks: grp, grp + ngrp, ...
        auto prefetch = [&](int mb) {
          const int c0 = (grp + mb * ngrp) * bw;
          float* dst = pf + (mb % (PD + 1)) * PS;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int pt = c0 + j;
            const float* src = Kp;
            bool v = lv && pt < n;
            if (phase == 2) {
              v = v && pt > 0 && pt < n - 1 && ((cls == kLineInterior && !first) || cls == kLineCopyU);
              src = cls == kLineCopyU ? up : outp;
            }
            cp_async4(dst + j * 32 + lane, (v ? src : Kp) + (v ? lb + pt * stride : 0), v);
          }
          cp_async_commit();
        };
        for (int pb = 0; pb < PD && pb < nmy; ++pb) prefetch(pb);
        for (int mb = 0; mb < nmy; ++mb) {
          const int c0 = (grp + mb * ngrp) * bw;
          if (mb + PD < nmy) {
            prefetch(mb + PD);
            cp_async_wait<PD>();
          } else if (nmy - 1 - mb >= 1) {
            cp_async_wait<1>();
          } else {
            cp_async_wait<0>();
          }
          const float* cur = pf + (mb % (PD + 1)) * PS;
          float v[16];
          if (c0 < nA) {
            tmem_ld16(tl + (uint32_t)c0, v);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = (xend && c0 + j == n - 1) ? gl : 0.f;
          }
          if (phase == 1) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (c0 + j == 0) e0 = v[j];
              if (c0 + j == n - 1) eN = v[j];
            }
          }
          if (lv) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int pt = c0 + j;
              const int idx = lb + pt * stride;
              const float ld = cur[j * 32 + lane];
              if (phase == 1) {
                if (pt < n) __stcg(Qp + idx, ld * v[j]);
              } else if (pt > 0 && pt < n - 1) {
                if (cls == kLineInterior) __stcg(outp + idx, ld - v[j]);
                else if (cls == kLineCopyU) __stcg(outp + idx, ld);
                else if (cls == kLineZero) __stcg(outp + idx, 0.f);
              }
            }
          }
        }
        // accumulator drained: hand it back to the MMA issuer
        tc_fence_before();
        mbar_arrive(tempty(b));
        if (phase == 1 && lv) {
          float* ef = reinterpret_cast<float*>(A.ends + L);
          if (grp == 0) ef[0] = e0;                        // point 0 is in block 0
          if (((n - 1) / bw) % ngrp == grp) ef[1] = eN;    // the block holding point n-1
        }
        if (phase == 2 && lv && grp == 0) line_ends(L, lb, stride, e0, eN);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(nbuf * tmem_cols)
                 : "memory");
  }
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
  if (!umma_ok(M, N, K) || (((uintptr_t)X | (uintptr_t)Wh | (uintptr_t)Wl) & 15) || !Wh) {
    set_error("umma_tf32x3_rot: unsupported shape or alignment");
    return CHEB_ERR_UNSUPPORTED;
  }
  const int n_tile = umma_n_tile(N);
  int tmem_cols = 32;
  while (tmem_cols < n_tile) tmem_cols *= 2;
  return chunk_k(Wl != nullptr) == 32 ? launch_rot<32>(X, Wh, Wl, Y, M, N, K, n_tile, tmem_cols, ep, s)
                         : launch_rot<16>(X, Wh, Wl, Y, M, N, K, n_tile, tmem_cols, ep, s);
}


// ---------------------------------------------------------------------------
// tensor-core route of the FP32 operator apply: per-plan resources
// ---------------------------------------------------------------------------
struct TensorApply {
  int nA1[3] = {0, 0, 0};   // phase-1 output columns (all n points), multiple of 16
  int nA2[3] = {0, 0, 0};   // phase-2 output columns (points 0 .. n-2)
  int Kp[3] = {0, 0, 0};    // padded K (points), multiple of 16
  float* Dh[3] = {nullptr, nullptr, nullptr};  // split-TF32 D, nA1 x Kp, zero padded
  float* Dl[3] = {nullptr, nullptr, nullptr};
  float* Dend[3] = {nullptr, nullptr, nullptr};  // row n-1 of D (FP32) when n = 257
  float* Q = nullptr;       // K * (D_a u), one field
  float2* ends = nullptr;   // per line: (D_a u) at both ends
  size_t ends_len = 0;
};

bool tensor_route_ok(const cheb_plan_s* p, int axis) {
  if (p->dim < 2 || axis < 0 || axis >= p->dim || has_flux(p)) return false;
  const int n = p->n[axis];
  return n >= 33 && n <= 257 && p->size() / (size_t)n >= (size_t)kBM;
}

static int tensor_setup(cheb_plan_s* p) {
  if (p->tap) return CHEB_OK;
  TensorApply* t = new TensorApply();
  auto fail = [&](int st) {
    tensor_apply_free(t);
    return st;
  };
  size_t maxl = 0;
  for (int a = 0; a < p->dim; ++a) {
    const int n = p->n[a];
    // n = 257: the MMA covers points 0..255; point 256 is a dot product in
    // the converters (so both phases keep two 256-column accumulators)
    t->nA1[a] = std::min(umma_n_tile(n), 256);
    t->nA2[a] = umma_n_tile(n - 1);
    t->Kp[a] = umma_n_tile(n);
    maxl = std::max(maxl, p->size() / (size_t)n);
    if (!tensor_route_ok(p, a)) continue;
    const std::vector<double> D = dense_deriv_matrix(n - 1, 2.0 / (p->hi[a] - p->lo[a]));
    const size_t rows = t->nA1[a], cols = t->Kp[a];
    std::vector<double> P(rows * cols, 0.0);
    for (int i = 0; i < std::min<int>(n, (int)rows); ++i)
      for (int j = 0; j < n; ++j) P[i * cols + j] = D[(size_t)i * n + j];
    if ((int)rows < n) {
      std::vector<float> de(cols, 0.f);
      for (int j = 0; j < n; ++j) de[j] = (float)D[(size_t)(n - 1) * n + j];
      if (cudaMalloc(&t->Dend[a], sizeof(float) * cols) != cudaSuccess) return fail(CHEB_ERR_NOMEM);
      if (cudaMemcpy(t->Dend[a], de.data(), sizeof(float) * cols, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(CHEB_ERR_CUDA);
    }
    std::vector<float> h(P.size()), l(P.size());
    tf32_split_host(P.data(), P.size(), h.data(), l.data());
    if (cudaMalloc(&t->Dh[a], sizeof(float) * P.size()) != cudaSuccess ||
        cudaMalloc(&t->Dl[a], sizeof(float) * P.size()) != cudaSuccess)
      return fail(CHEB_ERR_NOMEM);
    if (cudaMemcpy(t->Dh[a], h.data(), sizeof(float) * P.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->Dl[a], l.data(), sizeof(float) * P.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(CHEB_ERR_CUDA);
  }
  if (cudaMalloc(&t->Q, sizeof(float) * p->size()) != cudaSuccess ||
      cudaMalloc(&t->ends, sizeof(float2) * maxl) != cudaSuccess)
    return fail(CHEB_ERR_NOMEM);
  t->ends_len = maxl;
  p->tap = t;
  return CHEB_OK;
}

void tensor_apply_free(TensorApply* t) {
  if (!t) return;
  for (int a = 0; a < 3; ++a) {
    cudaFree(t->Dh[a]);
    cudaFree(t->Dl[a]);
    cudaFree(t->Dend[a]);
  }
  cudaFree(t->Q);
  cudaFree(t->ends);
  delete t;
}

template <bool XAX>
static int launch_dense(const CUtensorMap& mh, const CUtensorMap& ml, const LineGeo& lg, const DenseArgs& A,
                        int nA, cudaStream_t s) {
  const int nAx = dense_rows<XAX>(nA);
  int tmem_cols = 32;
  while (tmem_cols < nAx) tmem_cols *= 2;
  const int nbuf = 2 * tmem_cols <= 512 ? 2 : 1;
  int st;
  if ((st = ensure_smem_attr((const void*)dense_pass_kernel<XAX>, dense_smem_bytes(256)))) return st;
  const int ntiles = (lg.nl + kBM - 1) / kBM;
  const int grid = std::min(ntiles, sm_count());
  dense_pass_kernel<XAX><<<grid, dense_threads<XAX>(), dense_smem_bytes(nAx), s>>>(mh, ml, lg, A, nA,
                                                                                  tmem_cols, nbuf);
  CHEB_LAUNCH_CHECK("dense_pass_kernel");
  return CHEB_OK;
}

int tensor_apply_pass(const cheb_plan_s* pc, int axis, bool first, const float* K, const float* u, float* out,
                      cudaStream_t s) {
  cheb_plan_s* p = const_cast<cheb_plan_s*>(pc);  // lazily built route resources
  if (!tensor_route_ok(p, axis)) {
    set_error("tensor route needs 33 <= n <= 257 on a 2-D or 3-D grid");
    return CHEB_ERR_UNSUPPORTED;
  }
  int st;
  if ((st = tensor_setup(p))) return st;
  TensorApply& t = *p->tap;
  LineGeo lg;
  lg.axis = axis;
  lg.nx = p->n[0];
  lg.ny = p->n[1];
  lg.n = p->n[axis];
  lg.nl = (int)(p->size() / (size_t)lg.n);
  DenseArgs A;
  A.g = p->geom();
  A.first = first ? 1 : 0;
  A.K = K;
  A.Q = t.Q;
  A.ends = t.ends;
  A.u = u;
  A.out = out;
  for (int phase = 1; phase <= 2; ++phase) {
    const int nA = phase == 1 ? t.nA1[axis] : t.nA2[axis];
    CUtensorMap mh, ml;
    const int rows = axis == 0 ? dense_rows<true>(nA) : nA;  // D rows per stage (boxes of rows / 2)
    if ((st = make_map(&mh, t.Dh[axis], t.Kp[axis], t.nA1[axis], rows / 2, kDK))) return st;
    if ((st = make_map(&ml, t.Dl[axis], t.Kp[axis], t.nA1[axis], rows / 2, kDK))) return st;
    A.phase = phase;
    A.src = phase == 1 ? u : t.Q;
    A.Dend = phase == 1 ? t.Dend[axis] : nullptr;
    st = axis == 0 ? launch_dense<true>(mh, ml, lg, A, nA, s) : launch_dense<false>(mh, ml, lg, A, nA, s);
    if (st) return st;
  }
  return CHEB_OK;
}

int umma_wait_selftest(long long wait_cycles, cudaStream_t s) {
  if (wait_cycles < 1 || wait_cycles > kWaitCycles) { set_error("wait_cycles out of range"); return CHEB_ERR_ARG; }
  wait_selftest_kernel<<<1, 64, 0, s>>>(wait_cycles);
  CHEB_LAUNCH_CHECK("wait_selftest_kernel");
  CHEB_CUDA(cudaStreamSynchronize(s));
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
