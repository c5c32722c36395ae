// Solves of right-hand sides held in host memory (fem_fft_solve_host):
// upload, solve and download pipelined over CUDA streams owned by the plan.
// Host code.
//
// Two device slots (b, u) alternate between calls.  Call k uses slot k % 2:
//   upload stream:  wait (entry of call k on the caller's stream) and
//                   (solve of call k-2 done: slot b free) -> copy b -> ev_in
//   compute stream: wait ev_in, (download of call k-2 done: slot u free)
//                   -> fem_fft_solve(b slot -> u slot) -> ev_solved
//   download stream: wait ev_solved -> copy u -> ev_out
// so the upload of call k+1 and the download of call k-1 run under the
// solve of call k.  fem_fft_host_wait makes the caller's stream wait for
// every download issued so far.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "plan.h"

using namespace femfft;

namespace {

int host_setup(fem_fft_plan p) {
  if (p->hs_ready) return FEM_FFT_OK;
  const size_t bytes = (size_t)p->max_nrhs * p->dof * sizeof(double);
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc((void**)&p->hs_b[i], bytes) != cudaSuccess || cudaMalloc((void**)&p->hs_u[i], bytes) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("cudaMalloc of the host-solve slots failed");
      return FEM_FFT_ERR_OOM;
    }
    p->allocs.push_back(p->hs_b[i]);
    p->allocs.push_back(p->hs_u[i]);
    if (cudaEventCreateWithFlags(&p->hs_ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->hs_ev_solved[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->hs_ev_out[i], cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "host-solve events");
  }
  if (cudaEventCreateWithFlags(&p->hs_ev_entry, cudaEventDisableTiming) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "host-solve events");
  for (int i = 0; i < 3; ++i)
    if (cudaStreamCreateWithFlags(&p->hs_stream[i], cudaStreamNonBlocking) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "host-solve streams");
  p->hs_ready = 1;
  return FEM_FFT_OK;
}

}  // namespace

extern "C" {

int fem_fft_solve_host(fem_fft_plan p, const double* h_b, double* h_u, int64_t nrhs, void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;
  if (!p || !h_b || !h_u || nrhs < 0) return FEM_FFT_ERR_ARG;
  int rc = host_setup(p);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStream_t up = p->hs_stream[0], cmp = p->hs_stream[1], down = p->hs_stream[2];
  if (cudaEventRecord(p->hs_ev_entry, s) != cudaSuccess) return cuda_fail(cudaGetLastError(), "host solve");
  for (int64_t r0 = 0; r0 < nrhs; r0 += p->max_nrhs) {
    const int64_t cnt = std::min<int64_t>(p->max_nrhs, nrhs - r0);
    const size_t bytes = (size_t)cnt * p->dof * sizeof(double);
    const int k = p->hs_calls & 1;
    const bool reuse = p->hs_calls >= 2;
    cudaError_t e = cudaStreamWaitEvent(up, p->hs_ev_entry, 0);
    if (e == cudaSuccess && reuse) e = cudaStreamWaitEvent(up, p->hs_ev_solved[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->hs_b[k], h_b + (size_t)r0 * p->dof, bytes, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaEventRecord(p->hs_ev_in[k], up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cmp, p->hs_ev_in[k], 0);
    if (e == cudaSuccess && reuse) e = cudaStreamWaitEvent(cmp, p->hs_ev_out[k], 0);
    if (e != cudaSuccess) return cuda_fail(e, "host solve upload");
    rc = fem_fft_solve(p, p->hs_b[k], p->hs_u[k], cnt, cmp);
    if (rc && rc != FEM_FFT_ERR_NOT_CONVERGED) return rc;
    e = cudaEventRecord(p->hs_ev_solved[k], cmp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(down, p->hs_ev_solved[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_u + (size_t)r0 * p->dof, p->hs_u[k], bytes, cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess) e = cudaEventRecord(p->hs_ev_out[k], down);
    if (e != cudaSuccess) return cuda_fail(e, "host solve download");
    ++p->hs_calls;
  }
  return rc;
}

int fem_fft_host_wait(fem_fft_plan p, void* stream) {
  if (!p) return FEM_FFT_ERR_ARG;
  if (!p->hs_ready || p->hs_calls == 0) return FEM_FFT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < 2 && k < p->hs_calls; ++k)
    if (cudaStreamWaitEvent(s, p->hs_ev_out[k], 0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "host wait");
  return FEM_FFT_OK;
}

}  // extern "C"
