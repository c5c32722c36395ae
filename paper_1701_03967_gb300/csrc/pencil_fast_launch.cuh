// Launcher template of the register-radix pencil passes (pencil_fast.cuh).
#pragma once
#include "kernels.h"
#include "pencil_fast.cuh"

namespace femfft {

template <typename T, int NORD, int MODE, int V>
static int launch_fast_one(const FastParams& P, size_t smem, int threads, cudaStream_t s) {
  auto kern = pencil_fast_kernel<T, NORD, MODE, V>;
  const int e = ensure_dyn_smem((const void*)kern, smem);
  if (e) return e;
  // the prefetch distance: the CTAs resident at a time
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int& nsm = sms[dev >= 0 && dev < 64 ? dev : 0];
  if (!nsm && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 0;
  FastParams Pl = P;
  Pl.ahead = nsm * fast_min_blocks<V, MODE>();   // the CTAs resident at a time
  kern<<<(unsigned)P.g.tiles, threads, smem, s>>>(Pl);
  return (int)cudaGetLastError();
}

template <typename T, int V, int MODE>
static int launch_fast_mode(int n, const FastParams& P, size_t smem, int threads, cudaStream_t s) {
  switch (n) {
    case 1: return launch_fast_one<T, 1, MODE, V>(P, smem, threads, s);
    case 2: return launch_fast_one<T, 2, MODE, V>(P, smem, threads, s);
    case 3: return launch_fast_one<T, 3, MODE, V>(P, smem, threads, s);
    case 4: return launch_fast_one<T, 4, MODE, V>(P, smem, threads, s);
    case 5: return launch_fast_one<T, 5, MODE, V>(P, smem, threads, s);
    case 6: return launch_fast_one<T, 6, MODE, V>(P, smem, threads, s);
    case 7: return launch_fast_one<T, 7, MODE, V>(P, smem, threads, s);
    case 8: return launch_fast_one<T, 8, MODE, V>(P, smem, threads, s);
    case 9: return launch_fast_one<T, 9, MODE, V>(P, smem, threads, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template <typename T, int V>
static int launch_fast_v(int mode, int n, const FastParams& P, size_t smem, int threads, cudaStream_t s) {
  switch (mode) {
    case MODE_FWD: return launch_fast_mode<T, V, MODE_FWD>(n, P, smem, threads, s);
    case MODE_INV: return launch_fast_mode<T, V, MODE_INV>(n, P, smem, threads, s);
    case MODE_FUSED: return launch_fast_mode<T, V, MODE_FUSED>(n, P, smem, threads, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace femfft
