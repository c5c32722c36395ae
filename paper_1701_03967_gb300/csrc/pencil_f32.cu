// float32 instantiations of the pencil-pass kernels (mixed precision).
#include "pencil_launch.cuh"

namespace femfft {
int launch_pencil_f32(int mode, int n, const PassParams& P, size_t smem, int threads, cudaStream_t s) {
  return launch_pencil<float>(mode, n, P, smem, threads, s);
}
}  // namespace femfft
