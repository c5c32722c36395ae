// Stand-alone launches of algorithm (b) along axis 0 (device code in
// band.cuh): condensation, vertex solve and back substitution, one kernel each.
#include "band.cuh"

namespace femfft {

namespace {

template <typename T, int NORD>
__global__ void __launch_bounds__(kBandThreads) band_condense_kernel(BandParams P, int TW) {
  band_condense_block<T, NORD, false>(P, TW, blockIdx.x);
}
template <typename T, int NORD>
__global__ void __launch_bounds__(kBandThreads) band_vertex_kernel(BandParams P) {
  band_vertex_block<T, NORD, false>(P, blockIdx.x);
}
template <typename T, int NORD>
__global__ void __launch_bounds__(kBandThreads) band_back_kernel(BandParams P, int TW) {
  band_back_block<T, NORD, false>(P, TW, blockIdx.x);
}

template <typename T, int NORD>
int launch_band_n(const BandParams& P, cudaStream_t s) {
  const int TW = band_tw(P.inner);
  const long long blocks = band_elem_blocks(P, TW);
  band_condense_kernel<T, NORD><<<(unsigned)blocks, kBandThreads, 0, s>>>(P, TW);
  band_vertex_kernel<T, NORD><<<(unsigned)band_vertex_blocks(P), kBandThreads, 0, s>>>(P);
  band_back_kernel<T, NORD><<<(unsigned)blocks, kBandThreads, 0, s>>>(P, TW);
  return (int)cudaGetLastError();
}
template <typename T>
int launch_band_t(const BandParams& P, cudaStream_t s) {
  switch (P.n) {
    case 1: return launch_band_n<T, 1>(P, s);
    case 2: return launch_band_n<T, 2>(P, s);
    case 3: return launch_band_n<T, 3>(P, s);
    case 4: return launch_band_n<T, 4>(P, s);
    case 5: return launch_band_n<T, 5>(P, s);
    case 6: return launch_band_n<T, 6>(P, s);
    case 7: return launch_band_n<T, 7>(P, s);
    case 8: return launch_band_n<T, 8>(P, s);
    case 9: return launch_band_n<T, 9>(P, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace

int launch_band(const BandParams& P, bool f64, cudaStream_t s) {
  if (P.outer * P.inner <= 0 || P.K < 2) return 0;
  return f64 ? launch_band_t<double>(P, s) : launch_band_t<float>(P, s);
}

}  // namespace femfft
