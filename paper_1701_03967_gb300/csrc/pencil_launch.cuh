// Launcher template shared by pencil_f64.cu and pencil_f32.cu.
#pragma once
#include "kernels.h"
#include "pencil.cuh"

namespace femfft {

template <typename T, int NORD, int MODE, int WM>
static int launch_wm(const PassParams& P, size_t smem, int threads, cudaStream_t s) {
  auto kern = pencil_pass_kernel<T, NORD, MODE, WM>;
  const int e = ensure_dyn_smem((const void*)kern, smem);
  if (e) return e;
  kern<<<(unsigned)P.g.tiles, threads, smem, s>>>(P);
  return (int)cudaGetLastError();
}

// Small tiles (W <= kSmallW) use a variant whose per-thread pencil loops are
// bounded by kSmallW at compile time.
template <typename T, int NORD, int MODE>
static int launch_one(const PassParams& P, size_t smem, int threads, cudaStream_t s) {
  if (P.g.W <= kSmallW) return launch_wm<T, NORD, MODE, kSmallW>(P, smem, threads, s);
  return launch_wm<T, NORD, MODE, max_w<T>()>(P, smem, threads, s);
}

template <typename T, int MODE>
static int launch_mode(int n, const PassParams& P, size_t smem, int threads, cudaStream_t s) {
  switch (n) {
    case 1: return launch_one<T, 1, MODE>(P, smem, threads, s);
    case 2: return launch_one<T, 2, MODE>(P, smem, threads, s);
    case 3: return launch_one<T, 3, MODE>(P, smem, threads, s);
    case 4: return launch_one<T, 4, MODE>(P, smem, threads, s);
    case 5: return launch_one<T, 5, MODE>(P, smem, threads, s);
    case 6: return launch_one<T, 6, MODE>(P, smem, threads, s);
    case 7: return launch_one<T, 7, MODE>(P, smem, threads, s);
    case 8: return launch_one<T, 8, MODE>(P, smem, threads, s);
    case 9: return launch_one<T, 9, MODE>(P, smem, threads, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template <typename T>
static int launch_pencil(int mode, int n, const PassParams& P, size_t smem, int threads, cudaStream_t s) {
  switch (mode) {
    case MODE_FWD: return launch_mode<T, MODE_FWD>(n, P, smem, threads, s);
    case MODE_INV: return launch_mode<T, MODE_INV>(n, P, smem, threads, s);
    case MODE_FUSED: return launch_mode<T, MODE_FUSED>(n, P, smem, threads, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace femfft
