// Allocation-free operator apply: b = L u without a plan and without any
// device allocation.
//
// Who needs this: code that may not call cudaMalloc at the point where it
// applies the operator -- for example a host callback or custom-allocator
// hook that must not re-enter the allocator, a framework that forbids device
// allocation after its warm-up, or a process whose device memory is fully
// reserved by another allocator.  Such callers own the
// input and output buffers; the float64 temporaries of the axis-by-axis
// evaluation live in the fixed array below instead of plan workspace.
//
// Limits and sharing:
//  * The array holds kNoallocScratchBytes (64 MiB) on every GPU that loads
//    this library, for the life of the process.  A call needs
//    8 * DOF * T bytes, with DOF the unknowns of one right-hand side and
//    T = 0 (1D), 3 (2D) or 4 (3D) temporaries; larger problems (and 1D
//    problems above 9 * 2^20 unknowns) are rejected with FEM_FFT_ERR_ARG
//    before anything is launched, as are arguments plan creation rejects and
//    input and output ranges that overlap.  Right-hand sides are
//    processed one after the other through the same temporaries.
//  * All calls share the array and it keeps the contents of the last call.
//    Every temporary is completely written before it is read, so nothing has
//    to start at zero.  Calls whose kernels overlap on the GPU (different
//    streams, or different host threads) race on the array; serialise them.
//  * The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress, with that device current) and caches it; make
//    that first call before any stream capture begins.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/femfft.h"
#include "femfft_internal.h"
#include "kernels.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

// The scratch itself.  Host code must not take its address directly: the
// host-side symbol is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FEM_FFT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return FEM_FFT_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return FEM_FFT_OK;
}

using femfft::ApplyParams;

struct Ops {
  int N, n;
  long long M[femfft::kMaxN];
  int K[femfft::kMaxN];
  std::vector<double> A, C, Crow;
  double sa[femfft::kMaxN];   // a_i * 4 h_i^-2
  double c;
};

ApplyParams base_params(const Ops& o, int axis) {
  ApplyParams P;
  std::memset(&P, 0, sizeof(P));
  long long outer = 1, inner = 1;
  for (int j = 0; j < axis; ++j) outer *= o.M[j];
  for (int j = axis + 1; j < o.N; ++j) inner *= o.M[j];
  P.outer = outer;
  P.inner = inner;
  P.M = (int)o.M[axis];
  P.n = o.n;
  P.K = o.K[axis];
  return P;
}

// term t: alpha * (A if stiff else C) + beta * C, with exact row sums
void term(const Ops& o, ApplyParams& P, int t, bool stiff, double alpha, double beta, int src, int dst) {
  const int n1 = o.n + 1, n = o.n, R = n / 2 + 1, Pp = (n + 1) / 2, SP = Pp + 1;
  std::vector<double> M(n1 * n1);
  for (int i = 0; i < n1 * n1; ++i) M[i] = alpha * (stiff ? o.A[i] : o.C[i]) + beta * o.C[i];
  // even/odd halves (layout of the apply kernel)
  for (int q = 0; q < R; ++q) {
    for (int j = 0; j < Pp; ++j) {
      P.mats[t][q * SP + j] = 0.5 * (M[q * n1 + j] + M[q * n1 + (n - j)]);
      P.mats[t][R * SP + q * Pp + j] = 0.5 * (M[q * n1 + j] - M[q * n1 + (n - j)]);
    }
    P.mats[t][q * SP + Pp] = (n % 2 == 0) ? M[q * n1 + n / 2] : 0.0;
  }
  for (int r = 0; r < n1; ++r) P.rows1[t][r] = (stiff ? 0.0 : alpha * o.Crow[r]) + beta * o.Crow[r];
  P.t_src[t] = src;
  P.t_dst[t] = dst;
}

int launch(const ApplyParams& P, cudaStream_t s) {
  int e = femfft::launch_apply(P, s);
  return e ? FEM_FFT_ERR_CUDA : FEM_FFT_OK;
}

// b = L u for one right-hand side, temporaries X, Y, Z, W in the scratch.
// Same factorisation as the plan's operator apply (stiffness factors on u,
// mass factors afterwards).
int apply_one(const Ops& o, const double* u, double* b, double* X, double* Y, double* Z, double* W,
              cudaStream_t s) {
  int rc;
  if (o.N == 1) {
    ApplyParams P = base_params(o, 0);
    P.in[0] = u;
    P.out[0] = b;
    P.nterm = P.nout = 1;
    term(o, P, 0, true, o.sa[0], o.c, 0, 0);
    return launch(P, s);
  }
  {
    ApplyParams P = base_params(o, 0);          // X = (a1 s1 A + c C)_1 u
    P.in[0] = u;
    P.out[0] = X;
    P.nterm = P.nout = 1;
    term(o, P, 0, true, o.sa[0], o.c, 0, 0);
    if ((rc = launch(P, s))) return rc;
  }
  {
    ApplyParams P = base_params(o, 1);          // Y = C_2 X, Z = a2 s2 A_2 u
    P.in[0] = X;
    P.in[1] = u;
    P.out[0] = Y;
    P.out[1] = Z;
    P.nterm = P.nout = 2;
    term(o, P, 0, false, 1.0, 0.0, 0, 0);
    term(o, P, 1, true, o.sa[1], 0.0, 1, 1);
    if ((rc = launch(P, s))) return rc;
  }
  if (o.N == 2) {
    ApplyParams P = base_params(o, 0);          // b = Y + C_1 Z
    P.in[0] = Z;
    P.out[0] = b;
    P.addend = Y;
    P.nterm = P.nout = 1;
    term(o, P, 0, false, 1.0, 0.0, 0, 0);
    return launch(P, s);
  }
  {
    ApplyParams P = base_params(o, 0);          // Y += C_1 Z
    P.in[0] = Z;
    P.out[0] = Y;
    P.addend = Y;
    P.nterm = P.nout = 1;
    term(o, P, 0, false, 1.0, 0.0, 0, 0);
    if ((rc = launch(P, s))) return rc;
  }
  {
    ApplyParams P = base_params(o, 2);          // W = C_3 Y, X = a3 s3 A_3 u
    P.in[0] = Y;
    P.in[1] = u;
    P.out[0] = W;
    P.out[1] = X;
    P.nterm = P.nout = 2;
    term(o, P, 0, false, 1.0, 0.0, 0, 0);
    term(o, P, 1, true, o.sa[2], 0.0, 1, 1);
    if ((rc = launch(P, s))) return rc;
  }
  {
    ApplyParams P = base_params(o, 1);          // Z = C_2 X
    P.in[0] = X;
    P.out[0] = Z;
    P.nterm = P.nout = 1;
    term(o, P, 0, false, 1.0, 0.0, 0, 0);
    if ((rc = launch(P, s))) return rc;
  }
  ApplyParams P = base_params(o, 0);            // b = W + C_1 Z
  P.in[0] = Z;
  P.out[0] = b;
  P.addend = W;
  P.nterm = P.nout = 1;
  term(o, P, 0, false, 1.0, 0.0, 0, 0);
  return launch(P, s);
}

bool k_supported(int64_t K) {
  if (K < 2 || K > (1 << 20) || K % 2) return false;
  while (K % 2 == 0) K /= 2;
  while (K % 3 == 0) K /= 3;
  return K == 1;
}

}  // namespace

extern "C" int fem_fft_apply_noalloc(int N, int n, const int64_t* h_K, const double* h_X, const double* h_a,
                                     double c, const double* d_u, double* d_b, int64_t nrhs, void* stream) {
  if (N < 1 || N > femfft::kMaxN || n < 1 || n > femfft::kMaxOrder || !h_K || !h_X || !h_a || nrhs < 0)
    return FEM_FFT_ERR_ARG;
  Ops o;
  o.N = N;
  o.n = n;
  o.c = c;
  // The same validity rules as fem_fft_plan_create (L positive definite).
  // The unknown count is bounded while it is formed, so that no product of
  // the accepted extents can wrap around: a 1D problem has at most
  // 9 * 2^20 - 1 unknowns, and with temporaries the scratch size bounds it.
  const int ntmp = N == 1 ? 0 : (N == 2 ? 3 : 4);
  const long long dof_max = ntmp ? (long long)(kNoallocScratchBytes / (8 * (size_t)ntmp)) : (long long)9 << 20;
  long long dof = 1;
  double cmin = 0.0;
  for (int i = 0; i < N; ++i) {
    if (!k_supported(h_K[i]) || !(h_X[i] > 0.0) || !std::isfinite(h_X[i]) || !(h_a[i] > 0.0) ||
        !std::isfinite(h_a[i]))
      return FEM_FFT_ERR_ARG;
    o.K[i] = (int)h_K[i];
    o.M[i] = (long long)n * h_K[i] - 1;
    o.sa[i] = h_a[i] * 4.0 * (double)h_K[i] * (double)h_K[i] / (h_X[i] * h_X[i]);
    if (o.M[i] > dof_max / dof) return FEM_FFT_ERR_ARG;   // too large for the scratch
    dof *= o.M[i];
    cmin -= M_PI * M_PI * h_a[i] / (h_X[i] * h_X[i]);
  }
  if (!std::isfinite(c) || !(c > cmin)) return FEM_FFT_ERR_ARG;
  if (nrhs > (long long)(INT64_MAX / 8) / dof) return FEM_FFT_ERR_ARG;
  if (nrhs == 0) return FEM_FFT_OK;
  if (!d_u || !d_b) return FEM_FFT_ERR_ARG;
  // input and output ranges must be disjoint (the kernels read u while b is written)
  {
    const uintptr_t u0 = (uintptr_t)d_u, b0 = (uintptr_t)d_b;
    const uintptr_t len = (uintptr_t)(nrhs * dof) * sizeof(double);
    if (u0 < b0 + len && b0 < u0 + len) return FEM_FFT_ERR_ARG;
  }
  void* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  femfft::reference_matrices(n, &o.A, &o.C, &o.Crow);
  double* t = static_cast<double*>(scratch);
  double *X = t, *Y = t + dof, *Z = t + 2 * dof, *W = t + 3 * dof;
  cudaStream_t s = (cudaStream_t)stream;
  for (int64_t r = 0; r < nrhs; ++r) {
    if ((rc = apply_one(o, d_u + r * dof, d_b + r * dof, X, Y, Z, W, s))) return rc;
  }
  return FEM_FFT_OK;
}
