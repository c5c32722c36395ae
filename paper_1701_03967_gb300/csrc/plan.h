// The plan object and the host helpers shared by the plan API (api.cu) and
// the batched scheduler (batch.cu).  Host code.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/femfft.h"
#include "femfft_internal.h"
#include "kernels.h"
#include "pencil.cuh"
#include "pencil_fast.cuh"

namespace femfft {

struct DevTables {
  void* tw = nullptr;
  void* rot = nullptr;
  void* fwd = nullptr;
  void* fwdc = nullptr;   // forward maps of the direct F_n-transform
  void* inv = nullptr;
  void* mu = nullptr;
  // register-radix passes (pencil_fast.cuh); null when the axis is not eligible
  void* tw2 = nullptr;
  void* gmap = nullptr;
  void* invn = nullptr;
  void* muk = nullptr;
};

// One launch of a solve chain, recorded instead of launched: the batched
// scheduler replays the recorded chains of many plans inside one persistent
// kernel.  kind 0: pencil pass (pp, with the plan's own tile choice);
// kind 1: operator apply (ap).
struct RecordedOp {
  int kind;   // 0 pencil pass, 1 operator apply, 2 band solve (algorithm (b))
  int mode, axis;
  PassParams pp;
  ApplyParams ap;
  BandParams bp;
};

void set_last_error(const std::string& what);
int cuda_fail(cudaError_t e, const char* what);

// FFT schedule of length K with V values per thread: radix 3 passes first,
// then radix 8 (if 8 | V), 4 (if 4 | V) and 2, greedily.  Returns false when
// V does not divide K, exceeds kMaxV, or some radix needed does not divide V.
bool fft_schedule_v(int K, int V, int* npass, int* radix);
// The default schedule of the stand-alone passes (V = 8 for powers of two,
// 12 or 6 with a factor 3).
void fft_schedule(int K, int* V, int* npass, int* radix);

// Tile geometry of a pass for W pencils per tile.
void set_pass_tiles(PassParams& P, int W);

// Per-pass FFT index data of P's radix schedule (P.ax.K, P.npass, P.radix):
// prod = product of the earlier radices, its mask when a power of two (else
// -1), twiddle stride K / (prod * radix).
void set_fft_passes(PassParams& P);

// Complex values per pencil in shared memory for a tile of W pencils.  The
// strided tile loads and stores put W pencils times 32 / W rows in a warp;
// a pitch with 2 pitch = 32 / W (mod 32) banks (float; 16 / W in 8-byte
// units for double) puts them in disjoint bank ranges.  Where a warp spans
// several FFT sequences (K / V < 32) or W is 1, the pitch is odd instead.
// At most kPitchSlack above K * Q.
constexpr int kPitchSlack = 16;
int tile_pitch(int K, int Q, int V, int W, bool strided, int elem_bytes);

// A pencil pass over pencils too long for one CTA's shared memory
// (longpass.cu): global-memory four-step FFT path.  outer x inner pencils
// (inner: their element stride, 1 for the contiguous axis); f64: the pass's
// arithmetic.
int run_long_pass(fem_fft_plan p, int mode, int axis, long long outer, long long inner, const void* in,
                  bool in_f64, void* out, bool out_f64, bool accum, bool f64, int* nonfinite, cudaStream_t s);

// Records the mixed-precision solve of nrhs right-hand sides (b -> u, then
// `steps` refinement steps) as the plan would launch it.  nrhs must not
// exceed the plan's max_nrhs.  b and u may be placeholder addresses.
int record_mixed_solve(fem_fft_plan p, const double* b, double* u, long long nrhs, int steps,
                       std::vector<RecordedOp>* ops);

}  // namespace femfft

struct fem_fft_plan_s {
  int N = 0, n = 0, precision = 0;
  int64_t K[femfft::kMaxN] = {0, 0, 0}, M[femfft::kMaxN] = {0, 0, 0};
  double X[femfft::kMaxN] = {1, 1, 1}, a[femfft::kMaxN] = {1, 1, 1}, c = 0.0;
  int64_t max_nrhs = 1, dof = 0;
  femfft::AxisHost ax[femfft::kMaxN];
  femfft::DevTables t64[femfft::kMaxN], t32[femfft::kMaxN];
  int nax[femfft::kMaxN] = {0, 0, 0};  // element order of every axis (n: the common order, 0 if they differ)
  std::vector<double> Aref_ax[femfft::kMaxN], Cref_ax[femfft::kMaxN];   // element matrices per axis
  std::vector<double> Crow_ax[femfft::kMaxN];   // exact row sums of Cref_ax (those of Aref_ax are 0)
  float* w32 = nullptr;                // mixed workspace [max_nrhs][dof]
  double* tmp[4] = {nullptr, nullptr, nullptr, nullptr};   // float64 temporaries
  double* d_scalars = nullptr;         // device scalars (norms, dots)
  double rtol = 0.0;
  int max_iter = 2;
  int residual_df = 1;                 // refinement residual in double-float (1) or float64 (0)
  int last_iters = -1;
  double last_rel = -1.0;
  int smem_optin = 0;
  std::vector<void*> allocs;
  // when set, pencil passes and applies are appended here instead of launched
  std::vector<femfft::RecordedOp>* rec = nullptr;
  // tile shape (pencils per CTA W) and FFT values per thread V chosen by
  // fem_fft_plan_tune per [mode][axis][float64]; W = 0: the default heuristic
  struct Tuned {
    int W = 0, V = 0;
  };
  Tuned tuned[3][femfft::kMaxN][2];
  // float passes on the register-radix kernels (pencil_fast.cuh) where the
  // axis allows it; fem_fft_plan_tune picks, per [mode][axis], the faster of
  // them and the shared-memory Stockham kernels (fast_choice: -1 not tuned,
  // which means the register-radix kernels for K >= 512; 0 / 1) and their
  // pencils per tile (fast_W, 0: the heuristic)
  int fast_passes = 1;
  int fast_W[3][femfft::kMaxN] = {{0}};
  int fast_choice[3][femfft::kMaxN] = {{-1, -1, -1}, {-1, -1, -1}, {-1, -1, -1}};
  // forward passes read the direct F_n-transform maps (fem_fft_forward_fn)
  int use_fwdc = 0;
  // non-finite input detection: the first pass of a solve that reads the
  // caller's right-hand side (check_in) raises d_flag; the flag is copied to
  // pinned h_flag at the end of the solve (event flag_ev)
  int* d_flag = nullptr;
  int* h_flag = nullptr;
  cudaEvent_t flag_ev = nullptr;
  const void* check_in = nullptr;
  int last_status = 0;                 // FEM_FFT_OK or FEM_FFT_ERR_NOT_CONVERGED of the last solve
  // host-buffer solves (host.cu): two device slots, three streams
  int hs_ready = 0;
  long long hs_calls = 0;
  double* hs_b[2] = {nullptr, nullptr};
  double* hs_u[2] = {nullptr, nullptr};
  cudaEvent_t hs_ev_in[2] = {nullptr, nullptr}, hs_ev_solved[2] = {nullptr, nullptr},
              hs_ev_out[2] = {nullptr, nullptr}, hs_ev_entry = nullptr;
  cudaStream_t hs_stream[3] = {nullptr, nullptr, nullptr};
  // long contiguous pencils (longpass.cu): workspace of packed sequences
  void* long_ws = nullptr;
  size_t long_ws_bytes = 0;
  // algorithm (b) of Section 4 (fem_fft_set_algorithm): band-solve tables
  // per position of the later axes (float64 and float32 copies), the element
  // data and the vertex-solve scratch
  int algo = 0;                        // 0: algorithm (a), 1: algorithm (b)
  void* band_tab64 = nullptr;
  void* band_tab32 = nullptr;
  void* band_scr = nullptr;
  femfft::BandParams band_proto;
  // kernel timing (fem_fft_profile)
  struct ProfRec {
    cudaEvent_t a, b;
    int kind;
    double bytes, flops;
  };
  bool profiling = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> event_pool;
};
