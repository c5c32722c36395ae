// float64 instantiations of the pencil-pass kernels.
#include "pencil_launch.cuh"

namespace femfft {
int launch_pencil_f64(int mode, int n, const PassParams& P, size_t smem, int threads, cudaStream_t s) {
  return launch_pencil<double>(mode, n, P, smem, threads, s);
}
}  // namespace femfft
