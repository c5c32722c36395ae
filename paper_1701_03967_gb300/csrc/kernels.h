// Host-side declarations of the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include "femfft_internal.h"

namespace femfft {

struct PassParams;

// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes on
// the current device.  The limit is a per-device attribute: the largest value
// set is remembered per (kernel, device) under a lock, so that concurrent
// first launches and several GPUs are handled.  Returns a cudaError_t value.
int ensure_dyn_smem(const void* kernel, size_t smem);

// pencil passes (pencil_f64.cu / pencil_f32.cu): mode 0 forward, 1 inverse,
// 2 fused forward/divide/inverse.  Returns a cudaError_t value.
int launch_pencil_f64(int mode, int n, const PassParams& P, size_t smem, int threads, cudaStream_t s);
int launch_pencil_f32(int mode, int n, const PassParams& P, size_t smem, int threads, cudaStream_t s);

// register-radix passes (pencil_fast_*.cu), float32, V = 16 or 32 values per
// thread.  Returns a cudaError_t value.
struct FastParams;
int launch_fast_f32(int mode, int n, const FastParams& P, size_t smem, int threads, cudaStream_t s);

// Shared-memory layout of a register-radix tile (a bank-conflict model of
// the FFT exchanges and the map phase, evaluated on the host): the sequence
// order, the pencil pitch (complex values) and the swizzle of each
// intermediate buffer that minimise shared-memory wavefronts.
void fast_layout(int K, int Q, int Qp, int W, int V, int npass, const int* radix, int nthreads, int* order,
                 int* pitch, int* swz);

// Matrix-free float64 application of element-block operators along one axis
// (apply.cu).  Every term adds mats[t] (an (n+1)x(n+1) element matrix,
// row-major) applied along the axis to input src[t] into output dst[t].
constexpr int kApplyMaxTerms = 4;
constexpr int kApplyMaxIn = 3;
constexpr int kApplyMaxOut = 4;
constexpr int kApplyMatMax = (kMaxOrder + 1) * (kMaxOrder + 1);

struct ApplyParams {
  const double* in[kApplyMaxIn];
  double* out[kApplyMaxOut];     // float64 outputs (unused in dot mode)
  int nterm, nout;
  int t_src[kApplyMaxTerms], t_dst[kApplyMaxTerms];
  double mats[kApplyMaxTerms][kApplyMatMax];
  // exact row sums E (1..1)^T of every term matrix (the stiffness rows sum to
  // zero exactly; float64 rounding of A does not preserve that)
  double rows1[kApplyMaxTerms][kMaxOrder + 1];
  // output 0 = addend + sum of its terms (addend may alias out[0]: every
  // thread reads and writes only its own positions); residual form:
  // output 0 = base - (addend + sum) when base != null
  const double* addend;
  const double* base;
  float* out0_f32;               // if set, output 0 is written as float32 here
  double* norms;                 // if set: += ||out0||^2 (norms[0]), ||base||^2 (norms[1])
  // dot mode: dots[o] += sum_i dotv[i] * out_o[i]; nothing is written
  const double* dotv;
  double* dots;
  long long outer, inner;
  int M, n, K;
  // double-float arithmetic (df64.cuh): inputs with in_df[i] set, the
  // outputs and the addend are double-float fields stored as two float
  // planes (hi at the pointer, lo `plane` elements after it); other inputs
  // and base are float64 and are split on load
  int df;
  int in_df[kApplyMaxIn];
  long long plane;
  // 1: every field of the launch carries the two boundary nodes of the
  // operated axis (extent M + 2, fine index g stored at g + 1); element
  // loads read the boundary values there, outputs are the M interior rows.
  // 0: extent M, boundary values zero.  (outer / inner count the stored
  // positions of the other axes either way.)
  int gofs;
  // with gofs: outputs are known to vanish outside the boundary layers (one
  // element deep at each end of every axis), and the output fields start at
  // zero; a thread whose element and position lie outside them skips its
  // loads, products and stores.  bnd_M: interior extents of all axes.
  int bnd, bnd_N, bnd_axis;
  long long bnd_M[kMaxN];
  int bnd_n[kMaxN];              // element orders of all axes (layer depths)
  int hax;                       // host bookkeeping: the operated axis (kernels ignore it)
  // double-float apply only: 1 = the nterm (two) products are summed into
  // output 0 (nout = 1); each term keeps its own input t_src[t]
  int sum_terms;
  // double-float apply: input tiles of shared memory the launch provides
  // (0: one per staged input); outputs leave through the tiles when they fit
  int tile_cap;
};

// Tile width TW of the apply kernels (a block covers TW positions times
// nthreads / TW elements): up to 32 consecutive positions of the axes after
// the operated one; on the contiguous axis itself (inner == 1) TW lines of
// about K elements each (K rounded up to a power of two, at least 8), no
// more lines than there are -- TW > 1 with inner == 1 is the lines mode.
inline int apply_tile_w(long long inner, long long outer, int K, int nthreads) {
  int TW = 1;
  if (inner > 1) {
    while (TW * 2 <= 32 && TW * 2 <= inner) TW *= 2;
    return TW;
  }
  int TE = 8;
  while (TE < K && TE < nthreads) TE *= 2;
  TW = nthreads / TE;
  while (TW > 1 && TW / 2 >= outer) TW /= 2;
  return TW;
}
// blocks of an apply launch with tile width TW
inline long long apply_tile_blocks(long long inner, long long outer, int K, int TW, int nthreads) {
  const bool lines = inner == 1 && TW > 1;
  const long long npos = lines ? outer : inner;
  const int TE = nthreads / TW;
  return (lines ? 1 : outer) * ((npos + TW - 1) / TW) * ((K + TE - 1) / TE);
}

// Thread tid of block bx of an apply launch (the decode both apply kernels
// use, and fem_fft_apply_block_map on the host): element tile et = bx mod
// etiles, then position tile wt and outer index o.  Normal tiling: TW
// consecutive positions after the axis, thread -> (tid mod TW, tid div TW);
// lines mode (lines: inner == 1 with TW > 1): TW lines (outer indices),
// thread -> (tid div TE, tid mod TE).  valid: the thread has an element.
struct ApplyThread {
  bool lines, valid;
  int TE, tw, te, estep;
  long long npos, et, wt, o, w;
  int e;
};
__host__ __device__ inline ApplyThread apply_decode(long long bx, int tid, int TW, int nthreads, int K,
                                                    long long inner, long long outer, bool lines) {
  ApplyThread d;
  d.lines = lines;
  d.TE = nthreads / TW;
  d.npos = lines ? outer : inner;
  const long long wtiles = (d.npos + TW - 1) / TW;
  const long long etiles = (K + d.TE - 1) / d.TE;
  d.et = bx % etiles;
  bx /= etiles;
  d.wt = bx % wtiles;
  d.o = lines ? 0 : bx / wtiles;
  d.tw = lines ? tid / d.TE : tid % TW;
  d.te = lines ? tid % d.TE : tid / TW;
  d.estep = lines ? 1 : TW;   // thread-index distance to the next element of the same position
  d.w = d.wt * TW + d.tw;
  d.e = (int)(d.et * d.TE + d.te);
  d.valid = d.w < d.npos && d.e < K;
  return d;
}

// The double-float apply handles one or two outputs, term t writing output t,
// or two terms summed into one output (sum_terms); an addend, a residual
// base or a float32 output only with one output.
inline bool apply_df_form_ok(const ApplyParams& P) {
  if (P.dotv || P.nout < 1 || P.nout > 2 || P.gofs) return false;
  if (P.nout > 1 && (P.addend || P.base || P.out0_f32)) return false;
  if (P.sum_terms) {
    if (P.nout != 1 || P.nterm != 2) return false;
    return P.t_dst[0] == 0 && P.t_dst[1] == 0;
  }
  if (P.nterm != P.nout) return false;
  for (int t = 0; t < P.nterm; ++t)
    if (P.t_dst[t] != t) return false;
  return true;
}
// accumulators (template NOUT) of a double-float launch
inline int apply_df_nacc(const ApplyParams& P) { return P.sum_terms ? P.nterm : P.nout; }
int launch_apply(const ApplyParams& P, cudaStream_t s);
// Dirichlet data (dirichlet.cu): fields extended by the boundary node at
// each end of every axis (extents M_i + 2, C order, nrhs leading)
int launch_boundary_only(const double* g, double* gz, long long nrhs, int N, const long long* M, cudaStream_t s);
int launch_subtract_interior(double* b, const double* t, long long nrhs, int N, const long long* M, cudaStream_t s);
// y += a x over n float64 values (dirichlet.cu)
int launch_axpy(double* y, const double* x, double a, long long n, cudaStream_t s);

// Algorithm (b) along axis 0 (band.cu): the 1D problems
// [alpha calA + beta_w calC] v = y, one per position w of the later axes, on
// a field viewed as [outer][M][inner], in place.
constexpr int kBandMaxInt = kMaxOrder - 1;   // interior unknowns of an element
struct BandParams {
  void* f;             // the field (T = float or double), in place
  const void* tab;     // T [inner][n + 2]: beta, r_0..r_{n-2} = 1 / (alpha nu_m + beta), then
                       // sigma (off < 0) or D (off >= 0), then off (the vertex system below)
  void* scr;           // T [K - 1][outer * inner]: right-vertex contributions, then Thomas coefficients
  long long outer, inner;
  int M, K, n;
  double alpha;        // a_1 4 h_1^-2
  // element data: phi[i][l] (C_ii-orthonormal eigenvectors of A_ii phi = nu C_ii phi),
  // pta / ptc [l][b] = (phi^T A_ib / phi^T C_ib) for b = left, right vertex,
  // abi / cbi [b][m] = rows 0 and n of A / C over the interior columns
  double phi[kBandMaxInt * kBandMaxInt];
  double pta[kBandMaxInt][2], ptc[kBandMaxInt][2];
  double abi[2][kBandMaxInt], cbi[2][kBandMaxInt];
  float phif[kBandMaxInt * kBandMaxInt];
  float ptaf[kBandMaxInt][2], ptcf[kBandMaxInt][2];
  float abif[2][kBandMaxInt], cbif[2][kBandMaxInt];
};
int launch_band(const BandParams& P, bool f64, cudaStream_t s);

}  // namespace femfft
