// Line passes of the transform route for any N (the chirp form).  The DCT-I
// of a line is the length-2N DFT of its even extension (Sec. 2.2); when 2N
// is not a power of two that DFT runs as Bluestein's circular convolution
// of power-of-two length P = nextpow2(4N - 1), 8 .. 1024 (warp_dft_chirp).
// The passes are the generic line-pass kernel (same pass kinds, flux and
// boundary rows as the power-of-two passes) with 8-line tiles; the plan's
// tables hold the chirp and the transformed convolution kernel per axis.
#include "line_pass.cuh"

namespace cheb {

namespace {

constexpr int kChirpTL = 8;

template <typename T, int P, int CM>
int launch_chirp(const Geom& g, int axis, int kind, const AxisK<T>& ak, const T* K, const T* u, T* out,
                 cudaStream_t s, int nblocks, const T* C) {
  auto kern = line_pass_kernel<T, CHEB_ROUTE_TRANSFORM, P, CM, kChirpTL>;
  const size_t smem = pass_smem_bytes<T>(CHEB_ROUTE_TRANSFORM, ak.n, P, kChirpTL);
  int st;
  if ((st = ensure_smem_attr((const void*)kern, smem))) return st;
  kern<<<nblocks, kChirpTL * 16, smem, s>>>(g, axis, kind, ak, K, u, out, C);
  CHEB_LAUNCH_CHECK("line_pass_kernel (chirp)");
  return CHEB_OK;
}

}  // namespace

template <typename T>
int launch_chirp_pass(const Geom& g, int axis, int kind, const AxisK<T>& ak, int P, const T* K,
                      const T* u, T* out, cudaStream_t s, const T* C) {
  if (!ak.chirp || !ak.bhat || 4 * ak.N - 1 > P) {
    set_error("chirp pass without its tables");
    return CHEB_ERR_ARG;
  }
  int nblocks;
  if (axis == 0) nblocks = (g.n[1] * g.n[2] + kChirpTL - 1) / kChirpTL;
  else nblocks = ((g.n[0] + kChirpTL - 1) / kChirpTL) * (axis == 1 ? g.n[2] : g.n[1]);
  if (nblocks == 0) return CHEB_OK;
  // CM: elements per lane and parity class of the scans, ceil((N / 2 + 1) / 32)
  switch (P) {
    case 8: return launch_chirp<T, 8, 1>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 16: return launch_chirp<T, 16, 1>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 32: return launch_chirp<T, 32, 1>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 64: return launch_chirp<T, 64, 1>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 128: return launch_chirp<T, 128, 1>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 256: return launch_chirp<T, 256, 2>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 512: return launch_chirp<T, 512, 3>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    case 1024: return launch_chirp<T, 1024, 5>(g, axis, kind, ak, K, u, out, s, nblocks, C);
    default:
      set_error("chirp route needs a convolution length in [8, 1024]");
      return CHEB_ERR_UNSUPPORTED;
  }
}

template int launch_chirp_pass<double>(const Geom&, int, int, const AxisK<double>&, int, const double*,
                                       const double*, double*, cudaStream_t, const double*);
template int launch_chirp_pass<float>(const Geom&, int, int, const AxisK<float>&, int, const float*,
                                      const float*, float*, cudaStream_t, const float*);

}  // namespace cheb
