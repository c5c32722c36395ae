// Element-wise steps of the correction of f^h by non-zero Dirichlet data
// (Section 4 with u = g on the boundary): the boundary values of an extended
// field (every axis carries its two boundary nodes, extent M_i + 2) with the
// interior set to zero, and the subtraction of the interior of an extended
// field from an interior one.  The operator products between them are the
// float64 apply launches with gofs = 1.
#include <cuda_runtime.h>

#include "kernels.h"

namespace femfft {

namespace {

constexpr int kDirThreads = 256;

// extents of the extended field, axis N-1 fastest
struct ExtDims {
  int N;
  long long M[kMaxN];   // interior extents
};

__global__ void boundary_only_kernel(const double* __restrict__ g, double* __restrict__ gz, long long total,
                                     ExtDims d) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    bool interior = true;
    for (int ax = d.N - 1; ax >= 0; --ax) {
      const long long ext = d.M[ax] + 2;
      const long long i = r % ext;
      r /= ext;
      interior = interior && i >= 1 && i <= d.M[ax];
    }
    gz[idx] = interior ? 0.0 : g[idx];
  }
}

__global__ void subtract_interior_kernel(double* __restrict__ b, const double* __restrict__ t, long long total,
                                         ExtDims d) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    // interior multi-index -> extended offset (every index shifted by one)
    long long r = idx, off = 0, stride = 1;
    for (int ax = d.N - 1; ax >= 0; --ax) {
      const long long i = r % d.M[ax];
      r /= d.M[ax];
      off += (i + 1) * stride;
      stride *= d.M[ax] + 2;
    }
    off += r * stride;   // right-hand side index times the extended field size
    b[idx] -= t[off];
  }
}

ExtDims dims(int N, const long long* M) {
  ExtDims d;
  d.N = N;
  for (int i = 0; i < kMaxN; ++i) d.M[i] = i < N ? M[i] : 1;
  return d;
}

unsigned grid_for(long long total) {
  const long long want = (total + kDirThreads - 1) / kDirThreads;
  return (unsigned)(want < 152LL * 16 ? (want > 0 ? want : 1) : 152LL * 16);
}

}  // namespace

int launch_boundary_only(const double* g, double* gz, long long nrhs, int N, const long long* M, cudaStream_t s) {
  long long total = nrhs;
  for (int i = 0; i < N; ++i) total *= M[i] + 2;
  if (total <= 0) return 0;
  boundary_only_kernel<<<grid_for(total), kDirThreads, 0, s>>>(g, gz, total, dims(N, M));
  return (int)cudaGetLastError();
}

int launch_subtract_interior(double* b, const double* t, long long nrhs, int N, const long long* M, cudaStream_t s) {
  long long total = nrhs;
  for (int i = 0; i < N; ++i) total *= M[i];
  if (total <= 0) return 0;
  subtract_interior_kernel<<<grid_for(total), kDirThreads, 0, s>>>(b, t, total, dims(N, M));
  return (int)cudaGetLastError();
}

// y += a x over n float64 values (the tau b term of an implicit Euler
// right-hand side C u + tau b), grid-stride
__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, double a, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = fma(a, x[i], y[i]);
}

int launch_axpy(double* y, const double* x, double a, long long n, cudaStream_t s) {
  if (n <= 0) return (int)cudaSuccess;
  axpy_kernel<<<grid_for(n), kDirThreads, 0, s>>>(y, x, a, n);
  return (int)cudaGetLastError();
}

}  // namespace femfft
