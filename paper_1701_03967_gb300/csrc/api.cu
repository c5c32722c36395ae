// C ABI of the solver: plans, pass scheduling, solves, operator apply,
// refinement and gradient bilinear forms.  Host code.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "plan.h"

using namespace femfft;

namespace {

thread_local std::string g_last_error;

#define FEMFFT_CUDA(call, what)                      \
  do {                                               \
    cudaError_t e_ = (cudaError_t)(call);            \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

bool valid_K(int64_t K) {
  if (K < 2 || K > (1 << 20)) return false;
  if (K % 2) return false;
  while (K % 2 == 0) K /= 2;
  while (K % 3 == 0) K /= 3;
  return K == 1;
}

}  // namespace

namespace femfft {

void set_last_error(const std::string& what) { g_last_error = what; }

int ensure_dyn_smem(const void* kernel, size_t smem) {
  if (smem <= 48 * 1024) return (int)cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> enabled;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = enabled[std::make_pair(kernel, dev)];
  if (smem <= have) return (int)cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  have = smem;
  return (int)cudaSuccess;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return FEM_FFT_ERR_CUDA;
}

bool fft_schedule_v(int K, int V, int* npass, int* radix) {
  if (K < 2 || V < 2 || V > kMaxV || K % V) return false;
  int a = 0, b = 0, k = K;
  while (k % 2 == 0) { k /= 2; ++a; }
  while (k % 3 == 0) { k /= 3; ++b; }
  if (k != 1) return false;
  std::vector<int> r;
  if (b > 0 && V % 3) return false;
  for (int i = 0; i < b; ++i) r.push_back(3);
  while (a > 0) {
    int e = (a >= 3 && V % 8 == 0) ? 3 : (a >= 2 && V % 4 == 0) ? 2 : 1;
    if (V % 2) return false;
    r.push_back(1 << e);
    a -= e;
  }
  if ((int)r.size() > kMaxRadixPasses) return false;
  *npass = (int)r.size();
  for (size_t i = 0; i < r.size(); ++i) radix[i] = r[i];
  return true;
}

// Powers of two: radix 8 (then 4 or 2) with 8 values per thread; K with a
// factor 3: radix 3, then 4s with 12 values per thread (6 when K has a single
// factor 2).
void fft_schedule(int K, int* V, int* npass, int* radix) {
  int a = 0, k = K;
  while (k % 2 == 0) { k /= 2; ++a; }
  int v;
  if (k > 1) v = a >= 2 ? 12 : 6;
  else v = a >= 3 ? 8 : K;
  *V = v;
  fft_schedule_v(K, v, npass, radix);
}

int tile_pitch(int K, int Q, int V, int W, bool strided, int elem_bytes) {
  int pitch = pencil_pitch_min(K, Q);
  const int B = elem_bytes == 4 ? 32 : 16;   // bank-wide slots of one wavefront
  if (strided && K / V >= 32 && W >= 2 && W <= B / 2) {
    const int mod = B / 2, want = (B / (2 * W)) % mod;
    while (pitch % mod != want) ++pitch;
    return pitch;
  }
  if (pitch % 2 == 0) pitch += 1;
  return pitch;
}

void set_fft_passes(PassParams& P) {
  P.kshift = -1;
  if (P.ax.K >= 2 && (P.ax.K & (P.ax.K - 1)) == 0) {
    P.kshift = 0;
    while ((1 << P.kshift) < P.ax.K) ++P.kshift;
  }
  int prod = 1;
  for (int ps = 0; ps < kMaxRadixPasses; ++ps) {
    if (ps < P.npass) {
      P.pprod[ps] = prod;
      P.pmask[ps] = (prod & (prod - 1)) == 0 ? prod - 1 : -1;
      P.pstride[ps] = P.ax.K / (prod * P.radix[ps]);
      prod *= P.radix[ps];
    } else {
      P.pprod[ps] = 0;
      P.pmask[ps] = 0;
      P.pstride[ps] = 0;
    }
  }
}

void set_pass_tiles(PassParams& P, int W) {
  P.g.W = W;
  if (P.g.inner == 1) {
    P.g.tiles_inner = 1;
    P.g.tiles = (P.g.outer + W - 1) / W;
  } else {
    P.g.tiles_inner = (P.g.inner + W - 1) / W;
    P.g.tiles = P.g.outer * P.g.tiles_inner;
  }
}

}  // namespace femfft

namespace {

int dev_alloc(fem_fft_plan p, void** ptr, size_t bytes) {
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return FEM_FFT_ERR_OOM;
  }
  p->allocs.push_back(*ptr);
  return FEM_FFT_OK;
}

cudaEvent_t pool_event(fem_fft_plan p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with an event pair when profiling is on.
struct ProfScope {
  fem_fft_plan p;
  cudaStream_t s;
  fem_fft_plan_s::ProfRec rec;
  bool on;
  ProfScope(fem_fft_plan p_, cudaStream_t s_, int kind, double bytes, double flops) : p(p_), s(s_), on(p_->profiling) {
    if (!on) return;
    rec.a = pool_event(p);
    rec.b = pool_event(p);
    rec.kind = kind;
    rec.bytes = bytes;
    rec.flops = flops;
    cudaEventRecord(rec.a, s);
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(rec.b, s);
    p->prof.push_back(rec);
  }
};

template <typename T>
int upload(fem_fft_plan p, const std::vector<double>& v, void** dst, cudaStream_t s) {
  std::vector<T> tmp(v.begin(), v.end());
  int rc = dev_alloc(p, dst, tmp.size() * sizeof(T));
  if (rc) return rc;
  FEMFFT_CUDA(cudaMemcpyAsync(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, s), "upload");
  FEMFFT_CUDA(cudaStreamSynchronize(s), "upload sync");
  return FEM_FFT_OK;
}

template <typename T>
int upload_axis(fem_fft_plan p, const AxisHost& ax, DevTables* d, cudaStream_t s) {
  int rc;
  if ((rc = upload<T>(p, ax.tw, &d->tw, s))) return rc;
  if ((rc = upload<T>(p, ax.rot, &d->rot, s))) return rc;
  if ((rc = upload<T>(p, ax.fwd, &d->fwd, s))) return rc;
  if ((rc = upload<T>(p, ax.fwdc, &d->fwdc, s))) return rc;
  if ((rc = upload<T>(p, ax.inv, &d->inv, s))) return rc;
  if ((rc = upload<T>(p, ax.mu, &d->mu, s))) return rc;
  if (ax.fast_V) {
    if ((rc = upload<T>(p, ax.tw2, &d->tw2, s))) return rc;
    if ((rc = upload<T>(p, ax.gmap, &d->gmap, s))) return rc;
    if ((rc = upload<T>(p, ax.invn, &d->invn, s))) return rc;
    if ((rc = upload<T>(p, ax.muk, &d->muk, s))) return rc;
  }
  return FEM_FFT_OK;
}

// ------------------------------------------------------------ pencil passes

struct PassPlan {
  PassParams P;
  size_t smem;
  int threads;
};

// Pencils per CTA and the CTA grid for a pass over [outer][M][inner].
int plan_pass(fem_fft_plan p, int mode, int axis, long long outer, long long inner, bool f64, PassPlan* pp) {
  const int n = p->nax[axis], K = (int)p->K[axis], M = (int)p->M[axis];
  const int Q = n / 2 + 1;
  const size_t csize = f64 ? 2 * sizeof(double) : 2 * sizeof(float);
  PassParams& P = pp->P;
  std::memset(&P, 0, sizeof(P));
  fft_schedule(K, &P.V, &P.npass, P.radix);
  // per-pencil bound for the tile size; the pitch itself depends on W
  const size_t per_pen = (size_t)(pencil_pitch_min(K, Q) + kPitchSlack) * csize;
  const size_t tables = 2 * (size_t)K * csize;   // twiddles and rotations staged in shared memory
  // shared memory per CTA: float passes keep two CTAs resident per SM
  const size_t per_sm = 226 * 1024;
  const int ctas = (f64 || mode == MODE_FUSED) ? 1 : kPencilCtasPerSm;
  const size_t cta_budget = ctas == 1 ? (size_t)std::min(p->smem_optin, 220 * 1024)
                                      : std::min<size_t>(p->smem_optin, per_sm / ctas - 1024);
  if (cta_budget <= tables + per_pen) {
    g_last_error = "pencil does not fit in shared memory";
    return FEM_FFT_ERR_ARG;
  }
  const size_t budget = cta_budget - tables;
  long long wmax = (long long)(budget / per_pen);
  wmax = std::min<long long>(wmax, f64 ? kMaxW64 : kMaxW);
  if (wmax < 1) {
    g_last_error = "pencil does not fit in shared memory";
    return FEM_FFT_ERR_ARG;
  }
  const int threads = f64 ? kPencilThreads64 : kPencilThreads;
  // chunk tasks of the sequence build: W * K <= kMaxChunkTasks * threads
  wmax = std::min<long long>(wmax, (long long)kMaxChunkTasks * threads / K);
  if (wmax < 1 || K / P.V > threads) {
    g_last_error = "K too large for one CTA";
    return FEM_FFT_ERR_ARG;
  }
  long long W;
  if (inner == 1) {
    // keep at least ~2 CTAs per SM when possible
    long long want = std::max<long long>(1, outer / (2 * 152));
    W = std::min(wmax, want);
  } else {
    // strided pencils: a power of two (the tile loaders map thread -> pencil
    // by t mod W)
    long long lim = std::min<long long>(wmax, inner);
    W = 1;
    while (W * 2 <= lim) W *= 2;
    long long tiles = outer * ((inner + W - 1) / W);
    while (W > 1 && tiles < 2 * 152) {
      W /= 2;
      tiles = outer * ((inner + W - 1) / W);
    }
  }
  // tuned shape (fem_fft_plan_tune), clipped to what this pass admits
  const fem_fft_plan_s::Tuned& tu = p->tuned[mode][axis][f64 ? 1 : 0];
  if (tu.W > 0) {
    int np, rad[kMaxRadixPasses];
    if (fft_schedule_v(K, tu.V, &np, rad) && K / tu.V <= threads) {
      P.V = tu.V;
      P.npass = np;
      for (int i = 0; i < kMaxRadixPasses; ++i) P.radix[i] = i < np ? rad[i] : 0;
    }
    long long w = std::min<long long>(tu.W, wmax);
    if (inner > 1) {
      long long p2 = 1;
      while (p2 * 2 <= std::min(w, inner)) p2 *= 2;
      w = p2;
    }
    W = std::max<long long>(1, w);
  }
  P.g.outer = outer;
  P.g.inner = inner;
  P.g.M = M;
  set_pass_tiles(P, (int)W);
  P.pitch = tile_pitch(K, Q, P.V, (int)W, inner > 1, f64 ? 8 : 4);
  const DevTables& d = f64 ? p->t64[axis] : p->t32[axis];
  P.ax.n = n;
  P.ax.K = K;
  P.ax.M = M;
  set_fft_passes(P);
  P.ax.tw = d.tw;
  P.ax.rot = d.rot;
  P.ax.fwd = p->use_fwdc ? d.fwdc : d.fwd;
  P.ax.inv = d.inv;
  P.ax.mu = d.mu;
  pp->smem = (size_t)W * P.pitch * csize + tables;
  pp->threads = threads;
  return FEM_FFT_OK;
}

// Register-radix passes (pencil_fast.cuh): float32 plans, power-of-two K in
// [16, 1024].  Pencils per tile W: as many as the shared memory holds (a
// power of two for strided pencils), no more than keep about two tiles per
// SM, at most what the sequence build covers (W K <= 8 threads); a tuned W
// (fem_fft_plan_tune) replaces the heuristic.
struct FastPlan {
  FastParams P;
  size_t smem;
  int threads;
};

bool fast_possible(fem_fft_plan p, int mode, int axis, bool f64) {
  return p->fast_passes && !f64 && !p->rec && p->ax[axis].fast_V && p->t32[axis].gmap &&
         (mode == MODE_FWD || mode == MODE_INV || mode == MODE_FUSED);
}

// The register-radix kernels where they apply and were measured faster
// (fem_fft_plan_tune), else by default for K >= 512: on the short pencils of
// the 3D and batched workloads (K <= 128) the shared-memory Stockham kernels
// measured faster with the first register-radix launch shapes, and taking
// the register-radix kernels from K = 64 on by default later gained only 2 %
// on the batched workload.
bool fast_eligible(fem_fft_plan p, int mode, int axis, bool f64) {
  if (!fast_possible(p, mode, axis, f64)) return false;
  const int ch = p->fast_choice[mode][axis];
  return ch < 0 ? p->K[axis] >= 512 : ch == 1;
}

int plan_fast(fem_fft_plan p, int mode, int axis, long long outer, long long inner, int Wwant, FastPlan* fp) {
  const AxisHost& ax = p->ax[axis];
  const int n = ax.n, K = ax.K, Q = n / 2 + 1, Qp = Q | 1;
  const int threads = fast_threads_rt(ax.fast_V, mode);
  FastParams& P = fp->P;
  std::memset(&P, 0, sizeof(P));
  const size_t csize = 2 * sizeof(float);
  // shared memory per CTA: the share of one of the CTAs the kernel is compiled to keep per SM
  const int ctas = fast_ctas_rt(ax.fast_V, mode);
  const size_t budget = ctas >= 2 ? (size_t)std::min<size_t>(p->smem_optin, 224 * 1024 / ctas)
                                  : (size_t)std::min(p->smem_optin, 220 * 1024);
  long long wmax = (long long)(budget / ((size_t)(K * Qp + 16) * csize));
  wmax = std::min<long long>(wmax, std::min<long long>(kMaxW, (long long)kFastChunkTasks * threads / K));
  if (wmax < 1) return FEM_FFT_ERR_ARG;
  long long W;
  if (Wwant > 0) {
    W = std::min<long long>(Wwant, wmax);
  } else if (inner == 1) {
    W = std::min<long long>(wmax, std::max<long long>(1, outer / (2 * 152)));
  } else {
    W = std::min<long long>(wmax, inner);
    long long tiles = outer * ((inner + W - 1) / W);
    while (W > 1 && tiles < 2 * 152) {
      W /= 2;
      tiles = outer * ((inner + W - 1) / W);
    }
  }
  if (inner > 1) {
    long long p2 = 1;
    while (p2 * 2 <= W) p2 *= 2;
    W = p2;
  }
  P.g.outer = outer;
  P.g.inner = inner;
  P.g.M = (int)ax.M;
  P.g.W = (int)W;
  if (inner == 1) {
    P.g.tiles_inner = 1;
    P.g.tiles = (outer + W - 1) / W;
  } else {
    P.g.tiles_inner = (inner + W - 1) / W;
    P.g.tiles = outer * P.g.tiles_inner;
  }
  P.K = K;
  P.Qp = Qp;
  P.V = ax.fast_V;
  P.Tn = K / ax.fast_V;
  P.npass = ax.fast_npass;
  for (int s = 0; s < kFastMaxPass; ++s) {
    P.radix[s] = ax.fast_radix[s];
    P.lprod[s] = ax.fast_lprod[s];
    P.twofs[s] = ax.fast_twofs[s];
  }
  fast_layout(K, Q, Qp, (int)W, P.V, P.npass, P.radix, threads, &P.seq_order, &P.pitch, P.swz);
  if ((size_t)W * P.pitch * csize > budget) {   // the pitch slack of the bank model
    W = std::max<long long>(1, W - 1);
    if (inner > 1) {
      long long p2 = 1;
      while (p2 * 2 <= W) p2 *= 2;
      W = p2;
    }
    P.g.W = (int)W;
    if (inner == 1) {
      P.g.tiles_inner = 1;
      P.g.tiles = (outer + W - 1) / W;
    } else {
      P.g.tiles_inner = (inner + W - 1) / W;
      P.g.tiles = outer * P.g.tiles_inner;
    }
    fast_layout(K, Q, Qp, (int)W, P.V, P.npass, P.radix, threads, &P.seq_order, &P.pitch, P.swz);
  }
  const DevTables& d = p->t32[axis];
  P.tw2 = d.tw2;
  P.rot = d.rot;
  P.gmap = d.gmap;
  P.invn = d.invn;
  P.muk = d.muk;
  fp->smem = (size_t)W * P.pitch * csize;
  fp->threads = threads;
  return FEM_FFT_OK;
}

int run_fast(fem_fft_plan p, int mode, int axis, long long outer, long long inner, const void* in, bool in_f64,
             void* out, bool out_f64, bool accum, cudaStream_t s) {
  FastPlan fp;
  int rc = plan_fast(p, mode, axis, outer, inner, p->fast_W[mode][axis], &fp);
  if (rc) return rc;
  FastParams& P = fp.P;
  P.in = in;
  P.out = out;
  P.nonfinite = (in_f64 && in == p->check_in) ? p->d_flag : nullptr;
  P.in_f64 = in_f64;
  P.out_f64 = out_f64;
  P.accum = accum;
  if (mode == MODE_FUSED) {
    P.dv.c = p->c;
    P.dv.nother = p->N - 1;
    for (int j = 1; j < p->N; ++j) {
      P.dv.Mo[j - 1] = p->M[j];
      P.dv.mu_o[j - 1] = p->t32[j].mu;
    }
  }
  const double elems = (double)outer * P.g.M * inner;
  const double bytes = elems * ((in_f64 ? 8 : 4) + (out_f64 ? 8 : 4) * (accum ? 2 : 1));
  const int kind = mode == MODE_FWD ? 0 : (mode == MODE_FUSED ? 1 : 2);
  int e;
  {
    ProfScope scope(p, s, kind, bytes, 0.0);
    e = launch_fast_f32(mode, p->nax[axis], P, fp.smem, fp.threads, s);
  }
  if (e) return cuda_fail((cudaError_t)e, "pencil pass launch");
  return FEM_FFT_OK;
}

int run_pass(fem_fft_plan p, int mode, int axis, long long nrhs, bool f64, const void* in, bool in_f64,
             void* out, bool out_f64, bool accum, cudaStream_t s) {
  long long outer = nrhs, inner = 1;
  for (int j = 0; j < axis; ++j) outer *= p->M[j];
  for (int j = axis + 1; j < p->N; ++j) inner *= p->M[j];
  if (fast_eligible(p, mode, axis, f64))
    return run_fast(p, mode, axis, outer, inner, in, in_f64, out, out_f64, accum, s);
  PassPlan pp;
  int rc = plan_pass(p, mode, axis, outer, inner, f64, &pp);
  if (rc == FEM_FFT_ERR_ARG && !p->rec) {
    // a pencil too long for one CTA: the global four-step path
    const double elems = (double)outer * p->M[axis] * inner;
    const double bytes = elems * ((in_f64 ? 8 : 4) + (out_f64 ? 8 : 4) * (accum ? 2 : 1));
    const int kind = mode == MODE_FWD ? 0 : (mode == MODE_FUSED ? 1 : 2);
    ProfScope scope(p, s, kind, bytes, 0.0);
    return run_long_pass(p, mode, axis, outer, inner, in, in_f64, out, out_f64, accum, f64,
                         (in_f64 && in == p->check_in) ? p->d_flag : nullptr, s);
  }
  if (rc) return rc;
  PassParams& P = pp.P;
  P.in = in;
  P.out = out;
  P.nonfinite = (in_f64 && in == p->check_in && !p->rec) ? p->d_flag : nullptr;
  P.in_f64 = in_f64;
  P.out_f64 = out_f64;
  P.accum = accum;
  if (mode == MODE_FUSED) {
    P.dv.c = p->c;
    P.dv.nother = p->N - 1;
    for (int j = 1; j < p->N; ++j) {
      P.dv.Mo[j - 1] = p->M[j];
      P.dv.mu_o[j - 1] = f64 ? p->t64[j].mu : p->t32[j].mu;
    }
  }
  if (p->rec) {
    RecordedOp op;
    std::memset(&op, 0, sizeof(op));
    op.kind = 0;
    op.mode = mode;
    op.axis = axis;
    op.pp = P;
    p->rec->push_back(op);
    return FEM_FFT_OK;
  }
  const double elems = (double)outer * P.g.M * inner;
  const double bytes = elems * ((in_f64 ? 8 : 4) + (out_f64 ? 8 : 4) * (accum ? 2 : 1));
  const int kind = mode == MODE_FWD ? 0 : (mode == MODE_FUSED ? 1 : 2);
  int e;
  {
    ProfScope scope(p, s, kind, bytes, 0.0);
    e = f64 ? launch_pencil_f64(mode, p->nax[axis], P, pp.smem, pp.threads, s)
            : launch_pencil_f32(mode, p->nax[axis], P, pp.smem, pp.threads, s);
  }
  if (e) return cuda_fail((cudaError_t)e, "pencil pass launch");
  return FEM_FFT_OK;
}

// Algorithm (b) along axis 0, in place on the work array (N >= 2).
int run_band(fem_fft_plan p, long long nrhs, bool f64, void* work, cudaStream_t s) {
  BandParams B = p->band_proto;
  B.f = work;
  B.tab = f64 ? p->band_tab64 : p->band_tab32;
  B.scr = p->band_scr;
  B.outer = nrhs;
  if (p->rec) {
    RecordedOp op;
    std::memset(&op, 0, sizeof(op));
    op.kind = 2;
    op.mode = f64 ? 1 : 0;
    op.bp = B;
    p->rec->push_back(op);
    return FEM_FFT_OK;
  }
  const double elems = (double)nrhs * p->dof;
  // bytes of the three phases: field read + written twice, vertex rows twice
  const double bytes = elems * (f64 ? 8.0 : 4.0) * (4.0 + 4.0 / p->nax[0]);
  int e;
  {
    ProfScope scope(p, s, 1, bytes, 0.0);
    e = launch_band(B, f64, s);
  }
  if (e) return cuda_fail((cudaError_t)e, "band solve launch");
  return FEM_FFT_OK;
}

// Tables of algorithm (b): for every position w of the later axes
// beta_w = c + sum_{i>=1} a_i s_i lambda_i, r_m = 1 / (alpha nu_m + beta_w) and
// the vertex system of the element Schur complement (sigma or D, and off);
// element data from the interior eigenpairs of the reference matrices.
int build_band_tables(fem_fft_plan p, cudaStream_t s) {
  const int n = p->nax[0], n1 = n + 1, NI = n - 1;
  const std::vector<double>& A = p->Aref_ax[0];
  const std::vector<double>& C = p->Cref_ax[0];
  std::vector<double> nu, phi;
  if (interior_eig(n, &nu, &phi)) return FEM_FFT_ERR_ASSUMPTION_A;
  BandParams& B = p->band_proto;
  std::memset(&B, 0, sizeof(B));
  B.M = (int)p->M[0];
  B.K = (int)p->K[0];
  B.n = n;
  B.alpha = p->a[0] * 4.0 * p->K[0] * p->K[0] / (p->X[0] * p->X[0]);
  long long inner = 1;
  for (int j = 1; j < p->N; ++j) inner *= p->M[j];
  B.inner = inner;
  const int bi[2] = {0, n};
  for (int i = 0; i < NI * NI; ++i) {
    B.phi[i] = phi[i];
    B.phif[i] = (float)phi[i];
  }
  std::vector<double> pta(NI * 2), ptc(NI * 2);
  for (int l = 0; l < NI; ++l)
    for (int b = 0; b < 2; ++b) {
      double sa = 0.0, sc = 0.0;
      for (int i = 0; i < NI; ++i) {
        sa += phi[i * NI + l] * A[(i + 1) * n1 + bi[b]];
        sc += phi[i * NI + l] * C[(i + 1) * n1 + bi[b]];
      }
      pta[l * 2 + b] = sa;
      ptc[l * 2 + b] = sc;
      B.pta[l][b] = sa;
      B.ptc[l][b] = sc;
      B.ptaf[l][b] = (float)sa;
      B.ptcf[l][b] = (float)sc;
    }
  for (int b = 0; b < 2; ++b)
    for (int m = 0; m < NI; ++m) {
      B.abi[b][m] = A[bi[b] * n1 + (m + 1)];
      B.cbi[b][m] = C[bi[b] * n1 + (m + 1)];
      B.abif[b][m] = (float)B.abi[b][m];
      B.cbif[b][m] = (float)B.cbi[b][m];
    }
  // per position of the later axes
  const int RB = n + 2;
  std::vector<double> tab((size_t)inner * RB);
  for (long long w = 0; w < inner; ++w) {
    double beta = p->c;
    long long rem = w;
    for (int j = p->N - 1; j >= 1; --j) {
      const long long idx = rem % p->M[j];
      rem /= p->M[j];
      beta += p->ax[j].mu[idx];
    }
    double* t = &tab[(size_t)w * RB];
    t[0] = beta;
    // Vertex system of the element Schur complement S (bisymmetric):
    // tridiag(off, D, off) = 2 delta I - off tridiag(-1, 2, -1), with
    // off = S_01 and the row sum delta = S_00 + S_01.  Since A 1 = 0,
    // S 1 = beta (Crow_b - E_bi E_ii^-1 Crow_i): delta carries no terms of
    // size alpha, while D = S_00 + S_11 would be a difference of them (for the
    // lowest modes D and 2 |off| agree to many digits).  Long double for both.
    typedef long double ld;
    const ld al = (ld)B.alpha, be = (ld)beta;
    ld S01 = al * (ld)A[bi[0] * n1 + bi[1]] + be * (ld)C[bi[0] * n1 + bi[1]];
    std::vector<ld> pcrow(NI, 0.0L);   // Phi^T Crow_i
    for (int m = 0; m < NI; ++m) {
      ld acc = 0.0L;
      for (int i = 0; i < NI; ++i) acc += (ld)phi[i * NI + m] * (ld)p->Crow_ax[0][i + 1];
      pcrow[m] = acc;
    }
    ld rowc = (ld)p->Crow_ax[0][0];          // Crow_0 - E_0i E_ii^-1 Crow_i
    for (int m = 0; m < NI; ++m) {
      const ld r = 1.0L / (al * (ld)nu[m] + be);
      t[1 + m] = (double)r;
      const ld e0 = al * (ld)pta[m * 2] + be * (ld)ptc[m * 2];
      const ld e1 = al * (ld)pta[m * 2 + 1] + be * (ld)ptc[m * 2 + 1];
      S01 -= e0 * r * e1;
      rowc -= e0 * r * pcrow[m];
    }
    const ld delta = be * rowc;
    if (S01 < 0.0L) {
      t[n] = (double)(2.0L * delta / -S01);   // sigma: T = (-off) (sigma I + tridiag(-1, 2, -1))
    } else {
      t[n] = (double)(2.0L * delta - 2.0L * S01);   // D: strongly diagonally dominant here
    }
    t[n + 1] = (double)S01;
  }
  int rc;
  if (!p->band_tab64 && (rc = dev_alloc(p, &p->band_tab64, tab.size() * sizeof(double)))) return rc;
  if (!p->band_tab32 && (rc = dev_alloc(p, &p->band_tab32, tab.size() * sizeof(float)))) return rc;
  const size_t scr_elems = (size_t)p->max_nrhs * inner * (p->K[0] - 1);
  if (!p->band_scr && (rc = dev_alloc(p, &p->band_scr, std::max<size_t>(1, scr_elems) * sizeof(double)))) return rc;
  std::vector<float> tab32(tab.begin(), tab.end());
  FEMFFT_CUDA(cudaMemcpyAsync(p->band_tab64, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s),
              "band tables");
  FEMFFT_CUDA(cudaMemcpyAsync(p->band_tab32, tab32.data(), tab32.size() * sizeof(float), cudaMemcpyHostToDevice, s),
              "band tables");
  FEMFFT_CUDA(cudaStreamSynchronize(s), "band tables");
  return FEM_FFT_OK;
}

// Algorithm (a): forward passes on axes N-1..1, fused forward/divide/inverse
// on axis 0, inverse passes on axes 1..N-1.
int solve_chain(fem_fft_plan p, bool f64, const void* in, bool in_f64, void* work, void* out, bool accum,
                long long nrhs, cudaStream_t s) {
  const int N = p->N;
  int rc;
  const void* cur = in;
  bool cur_f64 = in_f64;
  for (int ax = N - 1; ax >= 1; --ax) {
    if ((rc = run_pass(p, MODE_FWD, ax, nrhs, f64, cur, cur_f64, work, f64, false, s))) return rc;
    cur = work;
    cur_f64 = f64;
  }
  // fused pass: the last pass of the chain when N == 1
  if (N == 1) return run_pass(p, MODE_FUSED, 0, nrhs, f64, cur, cur_f64, out, true, accum, s);
  if (p->algo == 1) {
    // algorithm (b): banded solves along x_1 in place of the transforms there
    if ((rc = run_band(p, nrhs, f64, work, s))) return rc;
  } else if ((rc = run_pass(p, MODE_FUSED, 0, nrhs, f64, cur, cur_f64, work, f64, false, s))) {
    return rc;
  }
  for (int ax = 1; ax < N; ++ax) {
    bool last = ax == N - 1;
    if ((rc = run_pass(p, MODE_INV, ax, nrhs, f64, work, f64, last ? out : work, last ? true : f64,
                       last ? accum : false, s)))
      return rc;
  }
  return FEM_FFT_OK;
}

// ----------------------------------------------------------- operator chains

// Algorithmic traffic and float64 flops of one apply launch: every input
// field read once, every output written once; per output position and term
// one row of an (n+1)x(n+1) element matrix (two at an element vertex), i.e.
// 2 (n+1)^2 / n flops per position and term on average.
int apply_launch(fem_fft_plan p, const ApplyParams& P, cudaStream_t s) {
  if (p->rec) {
    RecordedOp op;
    std::memset(&op, 0, sizeof(op));
    op.kind = 1;
    op.ap = P;
    p->rec->push_back(op);
    return 0;
  }
  const double elems = (double)P.outer * P.M * P.inner;
  int nin = 0;
  for (int i = 0; i < kApplyMaxIn; ++i) nin += P.in[i] != nullptr;
  double bytes = elems * 8.0 * nin;
  if (P.dotv) {
    bytes += elems * 8.0;
  } else {
    for (int j = 0; j < P.nout; ++j) bytes += elems * ((j == 0 && P.out0_f32) ? 4.0 : 8.0);
    if (P.base) bytes += elems * 8.0;
    if (P.addend) bytes += elems * 8.0;
  }
  // executed float64 flops of the even/odd element products (FMA = 2):
  // per element and term 2 R (P+1) + 2 R P (half-size products), 3 P + 1
  // (split), 2 R (combine) and 4 R for the constant response of mass terms
  const int n = P.n, R = n / 2 + 1, Pp = (n + 1) / 2;
  double per_elem = 0.0;
  for (int t = 0; t < P.nterm; ++t) {
    bool mass = false;
    for (int r = 0; r <= n; ++r) mass |= P.rows1[t][r] != 0.0;
    const int ns = (n % 2 == 0) ? Pp + 1 : Pp;
    per_elem += 2.0 * R * ns + 2.0 * R * Pp + 3.0 * Pp + 2 + 2.0 * R + (mass ? 2.0 * R : 0.0);
  }
  double flops = elems / n * per_elem;
  if (P.df) {
    // float32 operations of the double-float algorithm (df64.cuh counts:
    // df_add 11, df_fma 15, one Dot2 term 12, split of a float64 value 12)
    // per element and term: load/split of the n+1 values, the centre value,
    // the P sums and differences, the half-size products, the combination,
    // the constant response of mass terms and the accumulation
    double ops = 0.0;
    for (int t = 0; t < P.nterm; ++t) {
      bool mass = false;
      for (int r = 0; r <= n; ++r) mass |= P.rows1[t][r] != 0.0;
      const int ns = (n % 2 == 0) ? Pp + 1 : Pp;
      const bool split = !P.in_df[P.t_src[t]];
      ops += (split ? 12.0 * (n + 1) : 0.0) + 13.0 + 33.0 * Pp + (n % 2 == 0 ? 11.0 : 0.0) +
             12.0 * R * (ns + Pp) + 22.0 * R + (mass ? 30.0 * R : 0.0) + 11.0 * (n + 1);
    }
    flops = elems / n * ops;
  }
  ProfScope scope(p, s, P.df ? 4 : 3, bytes, flops);
  return launch_apply(P, s);
}

// Even/odd halves of a bisymmetric element matrix M ((n+1)^2) in the layout
// of the apply kernel: Es' (R x (P+1)) then Ea' (R x P), R = n/2 + 1,
// P = (n+1)/2, Es'[q][j] = (M[q][j] + M[q][n-j]) / 2 (j < n/2; column P: the
// middle node M[q][n/2] for even n, else 0), Ea'[q][j] = (M[q][j] - M[q][n-j]) / 2.
void pack_even_odd(const std::vector<double>& Mx, int n, double* out) {
  const int n1 = n + 1, R = n / 2 + 1, P = (n + 1) / 2, SP = P + 1;
  for (int q = 0; q < R; ++q) {
    for (int j = 0; j < P; ++j) {
      out[q * SP + j] = 0.5 * (Mx[q * n1 + j] + Mx[q * n1 + (n - j)]);
      out[R * SP + q * P + j] = 0.5 * (Mx[q * n1 + j] - Mx[q * n1 + (n - j)]);
    }
    out[q * SP + P] = (n % 2 == 0) ? Mx[q * n1 + n / 2] : 0.0;
  }
}

// Term t of an apply launch along axis P.hax: matrix alpha E + beta E2 where
// E, E2 name that axis's stiffness (kMatA) or mass (kMatC) element matrix
// (E2 = 0: none); its exact row sums are alpha (E 1) + beta (E2 1) with
// A 1 = 0 and C 1 = Crow.
enum { kMatNone = 0, kMatA = 1, kMatC = 2 };
void set_mat(fem_fft_plan p, ApplyParams& A, int t, int E, double alpha, int E2, double beta) {
  const int ax = A.hax;
  const std::vector<double>& Ar = p->Aref_ax[ax];
  const std::vector<double>& Cr = p->Cref_ax[ax];
  const std::vector<double>& Crow = p->Crow_ax[ax];
  const int n1 = p->nax[ax] + 1;
  std::vector<double> M(n1 * n1);
  const std::vector<double>& Em = E == kMatA ? Ar : Cr;
  const std::vector<double>& E2m = E2 == kMatA ? Ar : Cr;
  for (int i = 0; i < n1 * n1; ++i) M[i] = alpha * Em[i] + (E2 ? beta * E2m[i] : 0.0);
  pack_even_odd(M, n1 - 1, A.mats[t]);
  for (int r = 0; r < n1; ++r) {
    double v = E == kMatC ? alpha * Crow[r] : 0.0;
    if (E2 == kMatC) v += beta * Crow[r];
    A.rows1[t][r] = v;
  }
}

ApplyParams apply_base(fem_fft_plan p, int axis, long long nrhs) {
  ApplyParams A;
  std::memset(&A, 0, sizeof(A));
  long long outer = nrhs, inner = 1;
  for (int j = 0; j < axis; ++j) outer *= p->M[j];
  for (int j = axis + 1; j < p->N; ++j) inner *= p->M[j];
  A.outer = outer;
  A.inner = inner;
  A.M = (int)p->M[axis];
  A.n = p->nax[axis];
  A.K = (int)p->K[axis];
  A.hax = axis;
  return A;
}

// kind 0: out = L u (float64);  kind 1: r = b - L u (float32 into r32, norms
// optional).  In float64 every stiffness factor acts on u directly and the
// mass factors are applied to its result (apply.cuh says why):
//   1D: L u = E_1 u,  E_1 = a_1 s_1 A + c C
//   2D: L u = C_2 (E_1 u) + C_1 (a_2 s_2 A_2 u)
//   3D: L u = C_3 [C_2 (E_1 u) + C_1 (a_2 s_2 A_2 u)] + C_1 C_2 (a_3 s_3 A_3 u)
// The temporaries p->tmp hold the partial products.
// The double-float residual takes the short chain (below): in 3D four
// launches and seven products instead of six and eight, in 2D two launches
// instead of three at the same four products; its last launch sums its two
// products in one set of row sums (apply_kernel_df with SUMT).

int operator_chain(fem_fft_plan p, const double* u, long long nrhs, int kind, double* out, const double* b,
                   float* r32, double* norms, cudaStream_t s) {
  const int N = p->N;
  double s_[kMaxN];
  for (int i = 0; i < N; ++i) s_[i] = p->a[i] * 4.0 * p->K[i] * p->K[i] / (p->X[i] * p->X[i]);
  // residual in double-float: every temporary is a double-float field, u and
  // b are float64 fields split on load
  const bool dfr = kind == 1 && p->residual_df;
  auto dfify = [&](ApplyParams& P) {
    if (!dfr) return;
    P.df = 1;
    P.plane = nrhs * p->dof;
    for (int i = 0; i < kApplyMaxIn; ++i) P.in_df[i] = (P.in[i] && P.in[i] != u) ? 1 : 0;
  };
  auto finish = [&](ApplyParams& P) {
    if (kind == 0) {
      P.out[0] = out;
    } else {
      P.base = b;
      P.out0_f32 = r32;
      P.norms = norms;
    }
  };
  auto one = [&](int axis, const double* in, double* o, int E, double alpha, int E2, double beta) {
    ApplyParams P = apply_base(p, axis, nrhs);
    P.in[0] = in;
    P.nterm = 1;
    P.nout = 1;
    P.out[0] = o;
    set_mat(p, P, 0, E, alpha, E2, beta);
    return P;
  };
  int e;
  if (N == 1) {
    ApplyParams P = one(0, u, nullptr, kMatA, s_[0], kMatC, p->c);
    finish(P);
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
    return FEM_FFT_OK;
  }
  double *X = p->tmp[0], *Y = p->tmp[1], *Z = p->tmp[2], *W = p->tmp[3];
  if (dfr) {
    // the double-float residual starts on the last axis, so that its last
    // launch sums two products into r (two launches in 2D, four in 3D).  Its
    // stiffness factors on axes 0 (and 1) act on mass products (C_N u, ...):
    // their double-float rounding (about 2^-48 of the field, not the 2^-53
    // of float64 and then amplified) leaves the refined solution within
    // 1e-12 of the oracle (2D n = 9 K = 1024: 8.6e-13; 3D: 5.6e-13):
    //   X = C_N u, Y = E_N u (E_N = a_N s_N A_N + c C_N), along axis N-1;
    //   3D: Z = C_2 X, W = a_2 s_2 A_2 X, then W += C_2 Y, along axis 1;
    //   r = b - (a_1 s_1 A_1 Z' + C_1 W'), along axis 0,
    // with (Z', W') = (X, Y) in 2D and (Z, W) in 3D
    const int last = N - 1;
    auto pair_out = [&](int axis, const double* in, double* o0, int E0, double al0, int E0b, double be0, double* o1,
                        int E1, double al1, int E1b, double be1) {
      ApplyParams P = apply_base(p, axis, nrhs);   // o0 = M0 in, o1 = M1 in (one staged input)
      P.in[0] = in;
      P.nterm = 2;
      P.nout = 2;
      P.out[0] = o0;
      P.out[1] = o1;
      set_mat(p, P, 0, E0, al0, E0b, be0);
      P.t_src[0] = 0; P.t_dst[0] = 0;
      set_mat(p, P, 1, E1, al1, E1b, be1);
      P.t_src[1] = 0; P.t_dst[1] = 1;
      dfify(P);
      return apply_launch(p, P, s);
    };
    if ((e = pair_out(last, u, X, kMatC, 1.0, kMatNone, 0.0, Y, kMatA, s_[last], kMatC, p->c)))
      return cuda_fail((cudaError_t)e, "apply");
    const double *F0 = X, *F1 = Y;
    if (N == 3) {
      if ((e = pair_out(1, X, Z, kMatC, 1.0, kMatNone, 0.0, W, kMatA, s_[1], kMatNone, 0.0)))
        return cuda_fail((cudaError_t)e, "apply");
      ApplyParams P = one(1, Y, W, kMatC, 1.0, kMatNone, 0.0);                 // W += C_2 Y
      P.addend = W;
      dfify(P);
      if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
      F0 = Z;
      F1 = W;
    }
    ApplyParams P = apply_base(p, 0, nrhs);                                   // r = b - (s_1 A_1 F0 + C_1 F1)
    P.in[0] = F0;
    P.in[1] = F1;
    P.nterm = 2;
    P.nout = 1;
    P.sum_terms = 1;
    set_mat(p, P, 0, kMatA, s_[0], kMatNone, 0.0);
    P.t_src[0] = 0; P.t_dst[0] = 0;
    set_mat(p, P, 1, kMatC, 1.0, kMatNone, 0.0);
    P.t_src[1] = 1; P.t_dst[1] = 0;
    finish(P);
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
    return FEM_FFT_OK;
  }
  {
    ApplyParams P = one(0, u, X, kMatA, s_[0], kMatC, p->c);                   // X = E_1 u
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
  }
  {
    ApplyParams P = apply_base(p, 1, nrhs);                             // Y = C_2 X, Z = a2 s2 A_2 u
    P.in[0] = X;
    P.in[1] = u;
    P.nterm = 2;
    P.nout = 2;
    P.out[0] = Y;
    P.out[1] = Z;
    set_mat(p, P, 0, kMatC, 1.0, kMatNone, 0.0);
    P.t_src[0] = 0; P.t_dst[0] = 0;
    set_mat(p, P, 1, kMatA, s_[1], kMatNone, 0.0);
    P.t_src[1] = 1; P.t_dst[1] = 1;
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
  }
  if (N == 2) {
    ApplyParams P = one(0, Z, nullptr, kMatC, 1.0, kMatNone, 0.0);          // L u = Y + C_1 Z
    P.addend = Y;
    finish(P);
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
    return FEM_FFT_OK;
  }
  {
    ApplyParams P = one(0, Z, Y, kMatC, 1.0, kMatNone, 0.0);                 // Y += C_1 Z
    P.addend = Y;
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
  }
  {
    ApplyParams P = apply_base(p, 2, nrhs);                             // W = C_3 Y, X = a3 s3 A_3 u
    P.in[0] = Y;
    P.in[1] = u;
    P.nterm = 2;
    P.nout = 2;
    P.out[0] = W;
    P.out[1] = X;
    set_mat(p, P, 0, kMatC, 1.0, kMatNone, 0.0);
    P.t_src[0] = 0; P.t_dst[0] = 0;
    set_mat(p, P, 1, kMatA, s_[2], kMatNone, 0.0);
    P.t_src[1] = 1; P.t_dst[1] = 1;
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
  }
  {
    ApplyParams P = one(1, X, Z, kMatC, 1.0, kMatNone, 0.0);                 // Z = C_2 X
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
  }
  {
    ApplyParams P = one(0, Z, nullptr, kMatC, 1.0, kMatNone, 0.0);          // L u = W + C_1 Z
    P.addend = W;
    finish(P);
    dfify(P);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
  }
  return FEM_FFT_OK;
}

// b -= L_full G on the interior nodes, G the boundary values of g (fields
// extended by the boundary node at each end of every axis): Section 4 with
// u = g on the boundary, f^h corrected by the data.  The chain of
// operator_chain (stiffness factors on G itself, mass factors after them),
// every launch on extended fields (gofs = 1) so that each product keeps the
// boundary positions of the other axes; the result's interior is subtracted
// from b.  Temporaries come from the stream-ordered allocator.
int dirichlet_chain(fem_fft_plan p, const double* g, double* b, long long nrhs, cudaStream_t s) {
  const int N = p->N;
  double s_[kMaxN];
  long long Mx[kMaxN];
  size_t ext = 1;
  for (int i = 0; i < N; ++i) {
    s_[i] = p->a[i] * 4.0 * p->K[i] * p->K[i] / (p->X[i] * p->X[i]);
    Mx[i] = p->M[i];
    ext *= (size_t)(p->M[i] + 2);
  }
  const size_t field = ext * (size_t)nrhs;
  const int nbuf = N == 1 ? 2 : (N == 2 ? 4 : 5);
  double* buf = nullptr;
  if (cudaMallocAsync(&buf, field * nbuf * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("dirichlet: temporaries");
    return FEM_FFT_ERR_OOM;
  }
  int rc = FEM_FFT_OK;
  double* Gz = buf;
  double* X = buf + field;
  double* Y = X + field;
  double* Z = Y + field;
  double* W = Z + field;
  auto ext_base = [&](int axis) {
    ApplyParams P = apply_base(p, axis, nrhs);
    long long outer = nrhs, inner = 1;
    for (int j = 0; j < axis; ++j) outer *= p->M[j] + 2;
    for (int j = axis + 1; j < N; ++j) inner *= p->M[j] + 2;
    P.outer = outer;
    P.inner = inner;
    P.gofs = 1;
    P.bnd = 1;   // the temporaries start at zero (memset below)
    P.bnd_N = N;
    P.bnd_axis = axis;
    for (int j = 0; j < N; ++j) {
      P.bnd_M[j] = p->M[j];
      P.bnd_n[j] = p->nax[j];
    }
    return P;
  };
  auto one = [&](int axis, const double* in, double* o, int E, double alpha, int E2, double beta) {
    ApplyParams P = ext_base(axis);
    P.in[0] = in;
    P.nterm = 1;
    P.nout = 1;
    P.out[0] = o;
    set_mat(p, P, 0, E, alpha, E2, beta);
    return P;
  };
  auto two = [&](int axis, const double* in0, double* o0, const double* in1, double* o1, double s1) {
    ApplyParams P = ext_base(axis);   // o0 = C in0, o1 = s1 A in1
    P.in[0] = in0;
    P.in[1] = in1;
    P.nterm = 2;
    P.nout = 2;
    P.out[0] = o0;
    P.out[1] = o1;
    set_mat(p, P, 0, kMatC, 1.0, kMatNone, 0.0);
    P.t_src[0] = 0; P.t_dst[0] = 0;
    set_mat(p, P, 1, kMatA, s1, kMatNone, 0.0);
    P.t_src[1] = 1; P.t_dst[1] = 1;
    return P;
  };
  auto run = [&](const ApplyParams& P) {
    if (rc) return;
    const int e = apply_launch(p, P, s);
    if (e) rc = cuda_fail((cudaError_t)e, "dirichlet apply");
  };
  double* T = X;
  int e = cudaMemsetAsync(buf, 0, field * nbuf * sizeof(double), s);
  if (!e) e = launch_boundary_only(g, Gz, nrhs, N, Mx, s);
  if (e) rc = cuda_fail((cudaError_t)e, "dirichlet boundary data");
  run(one(0, Gz, X, kMatA, s_[0], kMatC, p->c));               // X = E_1 G
  if (N >= 2) run(two(1, X, Y, Gz, Z, s_[1]));          // Y = C_2 X, Z = a2 s2 A_2 G
  if (N == 2) {
    ApplyParams P = one(0, Z, X, kMatC, 1.0, kMatNone, 0.0);  // T = Y + C_1 Z
    P.addend = Y;
    run(P);
  } else if (N == 3) {
    ApplyParams P = one(0, Z, Y, kMatC, 1.0, kMatNone, 0.0);  // Y += C_1 Z
    P.addend = Y;
    run(P);
    run(two(2, Y, W, Gz, X, s_[2]));                     // W = C_3 Y, X = a3 s3 A_3 G
    run(one(1, X, Z, kMatC, 1.0, kMatNone, 0.0));             // Z = C_2 X
    ApplyParams Q = one(0, Z, Y, kMatC, 1.0, kMatNone, 0.0);  // T = W + C_1 Z
    Q.addend = W;
    run(Q);
    T = Y;
  }
  if (!rc) {
    e = launch_subtract_interior(b, T, nrhs, N, Mx, s);
    if (e) rc = cuda_fail((cudaError_t)e, "dirichlet subtract");
  }
  cudaFreeAsync(buf, s);
  return rc;
}

// out = (prod_i calC_i) u: one mass application per axis, through the
// temporaries (float64).
int mass_chain(fem_fft_plan p, const double* u, long long nrhs, double* out, cudaStream_t s) {
  const int N = p->N;
  const double* cur = u;
  int e;
  for (int ax = 0; ax < N; ++ax) {
    ApplyParams P = apply_base(p, ax, nrhs);
    P.in[0] = cur;
    P.nterm = 1;
    P.nout = 1;
    double* dst = ax == N - 1 ? out : p->tmp[ax % 2];
    P.out[0] = dst;
    set_mat(p, P, 0, kMatC, 1.0, kMatNone, 0.0);
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
    cur = dst;
  }
  return FEM_FFT_OK;
}

// dots[i] += lam^T (dL/da_i) u (i < N), dots[N] += lam^T (dL/dc) u
int grad_chain(fem_fft_plan p, const double* u, const double* lam, long long nrhs, double* dots, cudaStream_t s) {
  const int N = p->N;
  double s_[kMaxN];
  for (int i = 0; i < N; ++i) s_[i] = 4.0 * p->K[i] * p->K[i] / (p->X[i] * p->X[i]);
  int e;
  if (N == 1) {
    ApplyParams P = apply_base(p, 0, nrhs);
    P.in[0] = u;
    P.nterm = 2;
    P.nout = 2;
    set_mat(p, P, 0, kMatA, s_[0], kMatNone, 0.0);
    P.t_src[0] = 0; P.t_dst[0] = 0;
    set_mat(p, P, 1, kMatC, 1.0, kMatNone, 0.0);
    P.t_src[1] = 0; P.t_dst[1] = 1;
    P.dotv = lam;
    P.dots = dots;
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
    return FEM_FFT_OK;
  }
  if (N == 2) {
    ApplyParams P = apply_base(p, 1, nrhs);       // t1 = C2 u, t2 = A2 u
    P.in[0] = u;
    P.nterm = 2;
    P.nout = 2;
    P.out[0] = p->tmp[0];
    P.out[1] = p->tmp[1];
    set_mat(p, P, 0, kMatC, 1.0, kMatNone, 0.0);
    P.t_src[0] = 0; P.t_dst[0] = 0;
    set_mat(p, P, 1, kMatA, 1.0, kMatNone, 0.0);
    P.t_src[1] = 0; P.t_dst[1] = 1;
    if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
    ApplyParams Q = apply_base(p, 0, nrhs);       // s1 A1 t1, s2 C1 t2, C1 t1
    Q.in[0] = p->tmp[0];
    Q.in[1] = p->tmp[1];
    Q.nterm = 3;
    Q.nout = 3;
    set_mat(p, Q, 0, kMatA, s_[0], kMatNone, 0.0);
    Q.t_src[0] = 0; Q.t_dst[0] = 0;
    set_mat(p, Q, 1, kMatC, s_[1], kMatNone, 0.0);
    Q.t_src[1] = 1; Q.t_dst[1] = 1;
    set_mat(p, Q, 2, kMatC, 1.0, kMatNone, 0.0);
    Q.t_src[2] = 0; Q.t_dst[2] = 2;
    Q.dotv = lam;
    Q.dots = dots;
    if ((e = apply_launch(p, Q, s))) return cuda_fail((cudaError_t)e, "apply");
    return FEM_FFT_OK;
  }
  ApplyParams P = apply_base(p, 2, nrhs);         // t = C3 u, v = A3 u
  P.in[0] = u;
  P.nterm = 2;
  P.nout = 2;
  P.out[0] = p->tmp[0];
  P.out[1] = p->tmp[1];
  set_mat(p, P, 0, kMatC, 1.0, kMatNone, 0.0);
  P.t_src[0] = 0; P.t_dst[0] = 0;
  set_mat(p, P, 1, kMatA, 1.0, kMatNone, 0.0);
  P.t_src[1] = 0; P.t_dst[1] = 1;
  if ((e = apply_launch(p, P, s))) return cuda_fail((cudaError_t)e, "apply");
  ApplyParams Q = apply_base(p, 1, nrhs);         // w1 = C2 t, w2 = A2 t
  Q.in[0] = p->tmp[0];
  Q.nterm = 2;
  Q.nout = 2;
  Q.out[0] = p->tmp[2];
  Q.out[1] = p->tmp[3];
  set_mat(p, Q, 0, kMatC, 1.0, kMatNone, 0.0);
  Q.t_src[0] = 0; Q.t_dst[0] = 0;
  set_mat(p, Q, 1, kMatA, 1.0, kMatNone, 0.0);
  Q.t_src[1] = 0; Q.t_dst[1] = 1;
  if ((e = apply_launch(p, Q, s))) return cuda_fail((cudaError_t)e, "apply");
  ApplyParams Q3 = apply_base(p, 1, nrhs);        // w3 = C2 v into tmp[0] (t is dead now)
  Q3.in[0] = p->tmp[1];
  Q3.nterm = 1;
  Q3.nout = 1;
  Q3.out[0] = p->tmp[0];
  set_mat(p, Q3, 0, kMatC, 1.0, kMatNone, 0.0);
  Q3.t_src[0] = 0; Q3.t_dst[0] = 0;
  if ((e = apply_launch(p, Q3, s))) return cuda_fail((cudaError_t)e, "apply");
  ApplyParams R = apply_base(p, 0, nrhs);         // s1 A1 w1, s2 C1 w2, s3 C1 w3, C1 w1
  R.in[0] = p->tmp[2];
  R.in[1] = p->tmp[3];
  R.in[2] = p->tmp[0];
  R.nterm = 4;
  R.nout = 4;
  set_mat(p, R, 0, kMatA, s_[0], kMatNone, 0.0);
  R.t_src[0] = 0; R.t_dst[0] = 0;
  set_mat(p, R, 1, kMatC, s_[1], kMatNone, 0.0);
  R.t_src[1] = 1; R.t_dst[1] = 1;
  set_mat(p, R, 2, kMatC, s_[2], kMatNone, 0.0);
  R.t_src[2] = 2; R.t_dst[2] = 2;
  set_mat(p, R, 3, kMatC, 1.0, kMatNone, 0.0);
  R.t_src[3] = 0; R.t_dst[3] = 3;
  R.dotv = lam;
  R.dots = dots;
  if ((e = apply_launch(p, R, s))) return cuda_fail((cudaError_t)e, "apply");
  return FEM_FFT_OK;
}

}  // namespace

namespace femfft {

int record_mixed_solve(fem_fft_plan p, const double* b, double* u, long long nrhs, int steps,
                       std::vector<RecordedOp>* ops) {
  if (!p || !ops || p->precision != FEM_FFT_MIXED || nrhs < 1 || nrhs > p->max_nrhs || steps < 0)
    return FEM_FFT_ERR_ARG;
  p->rec = ops;
  int rc = solve_chain(p, false, b, true, p->w32, u, false, nrhs, nullptr);
  for (int it = 0; it < steps && !rc; ++it) {
    rc = operator_chain(p, u, nrhs, 1, nullptr, b, p->w32, nullptr, nullptr);
    if (!rc) rc = solve_chain(p, false, p->w32, false, p->w32, u, true, nrhs, nullptr);
  }
  p->rec = nullptr;
  return rc;
}

}  // namespace femfft

// ====================================================================== ABI

extern "C" {

const char* fem_fft_strerror(int code) {
  switch (code) {
    case FEM_FFT_OK: return "ok";
    case FEM_FFT_ERR_ARG: return "invalid argument";
    case FEM_FFT_ERR_ASSUMPTION_A: return "1D eigenproblem failed (assumption (A))";
    case FEM_FFT_ERR_OOM: return "device out of memory";
    case FEM_FFT_ERR_CUDA: return "CUDA error";
    case FEM_FFT_ERR_TIMEOUT: return "device wait timed out";
    case FEM_FFT_ERR_NOT_CONVERGED: return "refinement did not converge";
    case FEM_FFT_ERR_NONFINITE: return "non-finite residual";
    default: return "unknown status";
  }
}

const char* fem_fft_last_error(void) { return g_last_error.c_str(); }

int fem_fft_plan_destroy(fem_fft_plan p) {
  if (!p) return FEM_FFT_ERR_ARG;
  cudaDeviceSynchronize();
  for (void* ptr : p->allocs) cudaFree(ptr);
  for (auto& r : p->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
  if (p->long_ws) cudaFree(p->long_ws);
  if (p->h_flag) cudaFreeHost(p->h_flag);
  if (p->flag_ev) cudaEventDestroy(p->flag_ev);
  for (int i = 0; i < 2; ++i) {
    if (p->hs_ev_in[i]) cudaEventDestroy(p->hs_ev_in[i]);
    if (p->hs_ev_solved[i]) cudaEventDestroy(p->hs_ev_solved[i]);
    if (p->hs_ev_out[i]) cudaEventDestroy(p->hs_ev_out[i]);
  }
  if (p->hs_ev_entry) cudaEventDestroy(p->hs_ev_entry);
  for (int i = 0; i < 3; ++i)
    if (p->hs_stream[i]) cudaStreamDestroy(p->hs_stream[i]);
  delete p;
  return FEM_FFT_OK;
}

int fem_fft_plan_create(fem_fft_plan* out, int N, int n, const int64_t* h_K, const double* h_X,
                        const double* h_a, double c, int precision, int64_t max_nrhs, void* stream) {
  if (N < 1 || N > kMaxN) {
    if (out) *out = nullptr;
    return FEM_FFT_ERR_ARG;
  }
  const int ns[kMaxN] = {n, n, n};
  return fem_fft_plan_create_orders(out, N, ns, h_K, h_X, h_a, c, precision, max_nrhs, stream);
}

int fem_fft_plan_create_orders(fem_fft_plan* out, int N, const int* h_n, const int64_t* h_K, const double* h_X,
                               const double* h_a, double c, int precision, int64_t max_nrhs, void* stream) {
  if (!out) return FEM_FFT_ERR_ARG;
  *out = nullptr;
  bool orders_ok = h_n != nullptr && N >= 1 && N <= kMaxN;
  for (int i = 0; orders_ok && i < N; ++i) orders_ok = h_n[i] >= 1 && h_n[i] <= kMaxOrder;
  if (!orders_ok || !h_K || !h_X || !h_a || max_nrhs < 1) {
    g_last_error = "argument out of range";
    return FEM_FFT_ERR_ARG;
  }
  if (precision != FEM_FFT_FP64 && precision != FEM_FFT_MIXED) return FEM_FFT_ERR_ARG;
  double cmin = 0.0;
  for (int i = 0; i < N; ++i) {
    if (!valid_K(h_K[i]) || !(h_X[i] > 0.0) || !(h_a[i] > 0.0) || !std::isfinite(h_X[i]) ||
        !std::isfinite(h_a[i])) {
      g_last_error = "K must be 2^p 3^q (p >= 1), X_i and a_i positive";
      return FEM_FFT_ERR_ARG;
    }
    cmin -= M_PI * M_PI * h_a[i] / (h_X[i] * h_X[i]);
  }
  if (!std::isfinite(c) || !(c > cmin)) {
    g_last_error = "c must exceed -pi^2 sum a_i / X_i^2";
    return FEM_FFT_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  fem_fft_plan p = new (std::nothrow) fem_fft_plan_s();
  if (!p) return FEM_FFT_ERR_OOM;
  p->N = N;
  p->n = h_n[0];
  for (int i = 0; i < N; ++i) {
    p->nax[i] = h_n[i];
    if (h_n[i] != h_n[0]) p->n = 0;   // no common order
  }
  p->precision = precision;
  p->c = c;
  p->max_nrhs = max_nrhs;
  p->dof = 1;
  for (int i = 0; i < N; ++i) {
    p->K[i] = h_K[i];
    p->X[i] = h_X[i];
    p->a[i] = h_a[i];
    p->M[i] = h_n[i] * h_K[i] - 1;
    p->dof *= p->M[i];
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (ce != cudaSuccess) {
    delete p;
    return cuda_fail(ce, "device query");
  }
  int rc = FEM_FFT_OK;
  for (int i = 0; i < N; ++i) reference_matrices(h_n[i], &p->Aref_ax[i], &p->Cref_ax[i], &p->Crow_ax[i]);
  for (int i = 0; i < N && !rc; ++i) {
    // identical axes share nothing on purpose: tables are small
    if (precompute_axis(h_n[i], (int)p->K[i], p->X[i], p->a[i], &p->ax[i])) rc = FEM_FFT_ERR_ASSUMPTION_A;
  }
  for (int i = 0; i < N && !rc; ++i) rc = upload_axis<double>(p, p->ax[i], &p->t64[i], s);
  if (precision == FEM_FFT_MIXED)
    for (int i = 0; i < N && !rc; ++i) rc = upload_axis<float>(p, p->ax[i], &p->t32[i], s);
  const size_t field = (size_t)max_nrhs * p->dof;
  if (!rc && precision == FEM_FFT_MIXED) rc = dev_alloc(p, (void**)&p->w32, field * sizeof(float));
  const int ntmp = N == 1 ? 0 : (N == 2 ? 3 : 4);
  for (int t = 0; t < ntmp && !rc; ++t) rc = dev_alloc(p, (void**)&p->tmp[t], field * sizeof(double));
  if (!rc) rc = dev_alloc(p, (void**)&p->d_scalars, 16 * sizeof(double));
  if (!rc) rc = dev_alloc(p, (void**)&p->d_flag, sizeof(int));
  if (!rc && cudaMallocHost((void**)&p->h_flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rc = FEM_FFT_ERR_OOM;
  }
  if (!rc && cudaEventCreateWithFlags(&p->flag_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    rc = FEM_FFT_ERR_CUDA;
  }
  if (!rc) {
    *p->h_flag = 0;
    if (cudaMemsetAsync(p->d_flag, 0, sizeof(int), s) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "flag");
  }
  if (rc) {
    for (void* ptr : p->allocs) cudaFree(ptr);
    if (p->h_flag) cudaFreeHost(p->h_flag);
    if (p->flag_ev) cudaEventDestroy(p->flag_ev);
    delete p;
    return rc;
  }
  *out = p;
  return FEM_FFT_OK;
}

int fem_fft_plan_set_coefficients(fem_fft_plan p, const double* h_a, double c, void* stream) {
  if (!p || !h_a) return FEM_FFT_ERR_ARG;
  double cmin = 0.0;
  for (int i = 0; i < p->N; ++i) {
    if (!(h_a[i] > 0.0) || !std::isfinite(h_a[i])) return FEM_FFT_ERR_ARG;
    cmin -= M_PI * M_PI * h_a[i] / (p->X[i] * p->X[i]);
  }
  if (!std::isfinite(c) || !(c > cmin)) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < p->N; ++i) {
    AxisHost& ax = p->ax[i];
    ax.a = h_a[i];
    for (int m = 0; m < ax.M; ++m) ax.mu[m] = ax.a * ax.s * ax.lam[m];
    fast_muk_update(&ax);
    if (ax.fast_V) {
      std::vector<float> k32(ax.muk.begin(), ax.muk.end());
      if (p->t64[i].muk)
        FEMFFT_CUDA(cudaMemcpyAsync(p->t64[i].muk, ax.muk.data(), ax.muk.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, s), "coefficients");
      if (p->t32[i].muk)
        FEMFFT_CUDA(cudaMemcpyAsync(p->t32[i].muk, k32.data(), k32.size() * sizeof(float), cudaMemcpyHostToDevice, s),
                    "coefficients");
    }
    std::vector<float> f32(ax.mu.begin(), ax.mu.end());
    FEMFFT_CUDA(cudaMemcpyAsync(p->t64[i].mu, ax.mu.data(), ax.M * sizeof(double), cudaMemcpyHostToDevice, s),
                "coefficients");
    if (p->t32[i].mu)
      FEMFFT_CUDA(cudaMemcpyAsync(p->t32[i].mu, f32.data(), ax.M * sizeof(float), cudaMemcpyHostToDevice, s),
                  "coefficients");
    FEMFFT_CUDA(cudaStreamSynchronize(s), "coefficients sync");
    p->a[i] = h_a[i];
  }
  p->c = c;
  if (p->algo == 1) return build_band_tables(p, s);
  return FEM_FFT_OK;
}

int fem_fft_set_residual_precision(fem_fft_plan p, int mode) {
  if (!p || (mode != FEM_FFT_RESIDUAL_F64 && mode != FEM_FFT_RESIDUAL_DF64)) return FEM_FFT_ERR_ARG;
  p->residual_df = mode == FEM_FFT_RESIDUAL_DF64 ? 1 : 0;
  return FEM_FFT_OK;
}

int fem_fft_set_refinement(fem_fft_plan p, double rtol, int max_iter) {
  if (!p || rtol < 0.0 || max_iter < 0) return FEM_FFT_ERR_ARG;
  p->rtol = rtol;
  p->max_iter = max_iter;
  return FEM_FFT_OK;
}

int fem_fft_last_info(fem_fft_plan p, int* iters, double* rel) {
  if (!p) return FEM_FFT_ERR_ARG;
  if (iters) *iters = p->last_iters;
  if (rel) *rel = p->last_rel;
  FEMFFT_CUDA(cudaEventSynchronize(p->flag_ev), "last solve");
  if (*p->h_flag) return FEM_FFT_ERR_NONFINITE;
  return p->last_status;
}

int fem_fft_plan_dims(fem_fft_plan p, int* N, int* n, int64_t* h_M, int* precision) {
  if (!p) return FEM_FFT_ERR_ARG;
  if (N) *N = p->N;
  if (n) *n = p->n;   // 0 when the axes have different orders (fem_fft_plan_orders)
  if (precision) *precision = p->precision;
  if (h_M)
    for (int i = 0; i < p->N; ++i) h_M[i] = p->M[i];
  return FEM_FFT_OK;
}

int fem_fft_plan_orders(fem_fft_plan p, int* h_n) {
  if (!p || !h_n) return FEM_FFT_ERR_ARG;
  for (int i = 0; i < p->N; ++i) h_n[i] = p->nax[i];
  return FEM_FFT_OK;
}

int fem_fft_axis_tables(fem_fft_plan p, int axis, double* h_lam, double* h_cnorm, double* h_p) {
  if (!p || axis < 0 || axis >= p->N) return FEM_FFT_ERR_ARG;
  const AxisHost& ax = p->ax[axis];
  if (h_lam) std::memcpy(h_lam, ax.lam.data(), ax.lam.size() * sizeof(double));
  if (h_cnorm) std::memcpy(h_cnorm, ax.cnorm.data(), ax.cnorm.size() * sizeof(double));
  if (h_p && ax.n > 1) std::memcpy(h_p, ax.pvec.data(), (size_t)ax.K * ax.n * (ax.n - 1) * sizeof(double));
  return FEM_FFT_OK;
}

int fem_fft_axis_precompute(int n, int64_t K, double X, double* h_lam, double* h_cnorm, double* h_p) {
  if (n < 1 || n > kMaxOrder || !valid_K(K) || !(X > 0.0)) return FEM_FFT_ERR_ARG;
  AxisHost ax;
  if (precompute_axis(n, (int)K, X, 1.0, &ax)) return FEM_FFT_ERR_ASSUMPTION_A;
  if (h_lam) std::memcpy(h_lam, ax.lam.data(), ax.lam.size() * sizeof(double));
  if (h_cnorm) std::memcpy(h_cnorm, ax.cnorm.data(), ax.cnorm.size() * sizeof(double));
  if (h_p && n > 1) std::memcpy(h_p, ax.pvec.data(), (size_t)K * n * (n - 1) * sizeof(double));
  return FEM_FFT_OK;
}

int fem_fft_profile(fem_fft_plan p, int enable) {
  if (!p) return FEM_FFT_ERR_ARG;
  if (!enable) {
    cudaDeviceSynchronize();
    for (auto& r : p->prof) {
      p->event_pool.push_back(r.a);
      p->event_pool.push_back(r.b);
    }
    p->prof.clear();
  }
  p->profiling = enable != 0;
  return FEM_FFT_OK;
}

int fem_fft_profile_read(fem_fft_plan p, int kind, int64_t* launches, double* ms, double* bytes, double* flops) {
  if (!p || kind < 0 || kind > 4) return FEM_FFT_ERR_ARG;
  int64_t cnt = 0;
  double t = 0, by = 0, fl = 0;
  for (auto& r : p->prof) {
    if (r.kind != kind) continue;
    FEMFFT_CUDA(cudaEventSynchronize(r.b), "profile sync");
    float dt = 0.f;
    FEMFFT_CUDA(cudaEventElapsedTime(&dt, r.a, r.b), "profile elapsed");
    ++cnt;
    t += dt;
    by += r.bytes;
    fl += r.flops;
  }
  if (launches) *launches = cnt;
  if (ms) *ms = t;
  if (bytes) *bytes = by;
  if (flops) *flops = fl;
  return FEM_FFT_OK;
}

int fem_fft_solve(fem_fft_plan p, const double* b, double* u, int64_t nrhs, void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;   // nothing to do (pointers may be NULL)
  if (!p || !b || !u || nrhs < 0) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const bool mixed = p->precision == FEM_FFT_MIXED;
  if (mixed && b == u && p->max_iter > 0) {
    g_last_error = "in-place mixed-precision solve needs max_iter = 0";
    return FEM_FFT_ERR_ARG;
  }
  // the first pass of every group raises d_flag on a non-finite b
  FEMFFT_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), s), "flag");
  p->last_status = FEM_FFT_OK;
  int rc = FEM_FFT_OK;
  for (int64_t r0 = 0; r0 < nrhs && !rc; r0 += p->max_nrhs) {
    const long long cnt = std::min<int64_t>(p->max_nrhs, nrhs - r0);
    const double* bb = b + (size_t)r0 * p->dof;
    double* uu = u + (size_t)r0 * p->dof;
    p->check_in = bb;
    if (!mixed) {
      rc = solve_chain(p, true, bb, true, uu, uu, false, cnt, s);
      p->check_in = nullptr;
      continue;
    }
    rc = solve_chain(p, false, bb, true, p->w32, uu, false, cnt, s);
    p->check_in = nullptr;
    if (rc) break;
    p->last_iters = 0;
    p->last_rel = -1.0;
    // with rtol > 0: the residual of every iterate is read back; when the
    // steps run out, the last iterate's residual is evaluated too, and a
    // value above rtol returns FEM_FFT_ERR_NOT_CONVERGED
    const int evals = p->rtol > 0.0 ? p->max_iter + 1 : p->max_iter;
    for (int it = 0; it < evals && !rc; ++it) {
      double* norms = nullptr;
      if (p->rtol > 0.0) {
        if ((rc = cudaMemsetAsync(p->d_scalars, 0, 2 * sizeof(double), s))) {
          rc = cuda_fail((cudaError_t)rc, "memset");
          break;
        }
        norms = p->d_scalars;
      }
      if ((rc = operator_chain(p, uu, cnt, 1, nullptr, bb, p->w32, norms, s))) break;
      if (norms) {
        double h[2];
        if (cudaMemcpyAsync(h, p->d_scalars, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          rc = cuda_fail(cudaGetLastError(), "norms");
          break;
        }
        if (!std::isfinite(h[0]) || !std::isfinite(h[1])) {
          rc = FEM_FFT_ERR_NONFINITE;
          break;
        }
        p->last_rel = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
        if (p->last_rel <= p->rtol) break;
        if (it == p->max_iter) {
          p->last_status = FEM_FFT_ERR_NOT_CONVERGED;
          break;
        }
      }
      if ((rc = solve_chain(p, false, p->w32, false, p->w32, uu, true, cnt, s))) break;
      p->last_iters = it + 1;
    }
  }
  p->check_in = nullptr;
  // the flag reaches the host with the stream (fem_fft_last_info waits for it)
  if (cudaMemcpyAsync(p->h_flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaEventRecord(p->flag_ev, s) != cudaSuccess) {
    if (!rc) rc = cuda_fail(cudaGetLastError(), "flag");
  }
  if (rc) return rc;
  return p->last_status;
}

int fem_fft_apply(fem_fft_plan p, const double* u, double* b, int64_t nrhs, void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;   // nothing to do (pointers may be NULL)
  if (!p || !u || !b || u == b || nrhs < 0) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  for (int64_t r0 = 0; r0 < nrhs; r0 += p->max_nrhs) {
    const long long cnt = std::min<int64_t>(p->max_nrhs, nrhs - r0);
    if ((rc = operator_chain(p, u + (size_t)r0 * p->dof, cnt, 0, b + (size_t)r0 * p->dof, nullptr, nullptr,
                             nullptr, s)))
      return rc;
  }
  return FEM_FFT_OK;
}

int fem_fft_apply_mass(fem_fft_plan p, const double* u, double* b, int64_t nrhs, void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;
  if (!p || !u || !b || u == b || nrhs < 0) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  for (int64_t r0 = 0; r0 < nrhs; r0 += p->max_nrhs) {
    const long long cnt = std::min<int64_t>(p->max_nrhs, nrhs - r0);
    if ((rc = mass_chain(p, u + (size_t)r0 * p->dof, cnt, b + (size_t)r0 * p->dof, s))) return rc;
  }
  return FEM_FFT_OK;
}

int fem_fft_dirichlet_rhs(fem_fft_plan p, const double* g, double* b, int64_t nrhs, void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;
  if (!p || !g || !b || nrhs < 0) return FEM_FFT_ERR_ARG;
  return dirichlet_chain(p, g, b, nrhs, (cudaStream_t)stream);
}

int fem_fft_set_algorithm(fem_fft_plan p, int algo, void* stream) {
  if (!p || (algo != FEM_FFT_ALGO_A && algo != FEM_FFT_ALGO_B)) return FEM_FFT_ERR_ARG;
  if (algo == FEM_FFT_ALGO_B) {
    if (p->N < 2) {
      g_last_error = "algorithm (b) needs N >= 2 (for N = 1 it is a single banded solve)";
      return FEM_FFT_ERR_ARG;
    }
    int rc = build_band_tables(p, (cudaStream_t)stream);
    if (rc) return rc;
  }
  p->algo = algo == FEM_FFT_ALGO_B ? 1 : 0;
  return FEM_FFT_OK;
}

int fem_fft_plan_tune(fem_fft_plan p, void* stream) {
  if (!p) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = p->precision == FEM_FFT_FP64;
  // scratch: the plan's own workspace, zeroed (contents do not affect timing)
  void* buf = f64 ? (void*)p->tmp[0] : (void*)p->w32;
  const size_t bytes = (size_t)p->max_nrhs * p->dof * (f64 ? sizeof(double) : sizeof(float));
  if (!buf) return FEM_FFT_OK;   // 1D FP64 plans have no temporary: nothing to tune against
  FEMFFT_CUDA(cudaMemsetAsync(buf, 0, bytes, s), "tune scratch");
  cudaEvent_t e0, e1;
  FEMFFT_CUDA(cudaEventCreate(&e0), "tune events");
  FEMFFT_CUDA(cudaEventCreate(&e1), "tune events");
  const bool was_profiling = p->profiling;
  p->profiling = false;
  int rc = FEM_FFT_OK;
  const int threads = f64 ? kPencilThreads64 : kPencilThreads;
  struct Pass { int mode, axis; };
  std::vector<Pass> passes;
  for (int ax = p->N - 1; ax >= 1; --ax) passes.push_back({MODE_FWD, ax});
  passes.push_back({MODE_FUSED, 0});
  for (int ax = 1; ax < p->N; ++ax) passes.push_back({MODE_INV, ax});
  for (const Pass& ps : passes) {
    float fast_best_ms = 1e30f;
    if (fast_possible(p, ps.mode, ps.axis, f64)) {
      p->fast_choice[ps.mode][ps.axis] = 1;
      // register-radix pass: pencils per tile W in 1, 2, 4, ... (the radix
      // schedule is fixed by K)
      int bestW = 0;
      float best_ms = 1e30f;
      long long outer = p->max_nrhs, inner = 1;
      for (int j = 0; j < ps.axis; ++j) outer *= p->M[j];
      for (int j = ps.axis + 1; j < p->N; ++j) inner *= p->M[j];
      for (int W = 1; W <= kMaxW && !rc; W *= 2) {
        FastPlan fp;
        if (plan_fast(p, ps.mode, ps.axis, outer, inner, W, &fp) || fp.P.g.W != W) continue;
        p->fast_W[ps.mode][ps.axis] = W;
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
          cudaEventRecord(e0, s);
          rc = run_pass(p, ps.mode, ps.axis, p->max_nrhs, f64, buf, f64, buf, f64, false, s);
          cudaEventRecord(e1, s);
          if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = FEM_FFT_ERR_CUDA;
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep > 0) ms = std::min(ms, t);
        }
        if (ms < best_ms) {
          best_ms = ms;
          bestW = W;
        }
      }
      p->fast_W[ps.mode][ps.axis] = bestW;   // 0: the heuristic
      fast_best_ms = best_ms;
      if (rc) break;
      p->fast_choice[ps.mode][ps.axis] = 0;   // now time the shared-memory kernels
    }
    fem_fft_plan_s::Tuned& tu = p->tuned[ps.mode][ps.axis][f64 ? 1 : 0];
    const int K = (int)p->K[ps.axis];
    fem_fft_plan_s::Tuned best;
    float best_ms = 1e30f;
    for (int V : {4, 8, 6, 12}) {
      int np, rad[kMaxRadixPasses];
      if (!fft_schedule_v(K, V, &np, rad) || K / V > threads) continue;
      for (int W = 1; W <= (f64 ? kMaxW64 : kMaxW); W *= 2) {
        tu.W = W;
        tu.V = V;
        // the candidate must keep its shape after clipping
        long long outer = p->max_nrhs, inner = 1;
        for (int j = 0; j < ps.axis; ++j) outer *= p->M[j];
        for (int j = ps.axis + 1; j < p->N; ++j) inner *= p->M[j];
        PassPlan pp;
        if (plan_pass(p, ps.mode, ps.axis, outer, inner, f64, &pp) || pp.P.g.W != W || pp.P.V != V) continue;
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
          cudaEventRecord(e0, s);
          rc = run_pass(p, ps.mode, ps.axis, p->max_nrhs, f64, buf, f64, buf, f64, false, s);
          cudaEventRecord(e1, s);
          if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = FEM_FFT_ERR_CUDA;
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep > 0) ms = std::min(ms, t);
        }
        if (rc) break;
        if (ms < best_ms) {
          best_ms = ms;
          best.W = W;
          best.V = V;
        }
      }
      if (rc) break;
    }
    tu = best;   // W = 0 (heuristic) if no candidate ran
    if (fast_possible(p, ps.mode, ps.axis, f64))
      p->fast_choice[ps.mode][ps.axis] = fast_best_ms <= best_ms ? 1 : 0;
    if (rc) break;
  }
  p->profiling = was_profiling;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int fem_fft_forward(fem_fft_plan p, const double* y, double* c, int64_t nrhs, void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;   // nothing to do (pointers may be NULL)
  if (!p || !y || !c || nrhs < 0) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  for (int ax = p->N - 1; ax >= 0; --ax) {
    if ((rc = run_pass(p, MODE_FWD, ax, nrhs, true, ax == p->N - 1 ? (const void*)y : (const void*)c, true, c,
                       true, false, s)))
      return rc;
  }
  return FEM_FFT_OK;
}

int fem_fft_heat_step(fem_fft_plan p, double tau, const double* u, const double* b, double* u_new, int64_t nrhs,
                      void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;
  if (!p || !u || !b || !u_new || u_new == u || u_new == b || nrhs < 0 || !(tau > 0.0) || !std::isfinite(tau))
    return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t total = (size_t)nrhs * p->dof;
  // the right-hand side C u + tau b is formed in u_new when the solve may run
  // in place, else in a stream-ordered temporary
  const bool in_place = p->precision == FEM_FFT_FP64 || p->max_iter == 0;
  double* rhs = u_new;
  if (!in_place) {
    cudaError_t e = cudaMallocAsync((void**)&rhs, total * sizeof(double), s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g_last_error = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
      return FEM_FFT_ERR_OOM;
    }
  }
  int rc = FEM_FFT_OK;
  for (int64_t r0 = 0; r0 < nrhs && !rc; r0 += p->max_nrhs) {
    const long long cnt = std::min<int64_t>(p->max_nrhs, nrhs - r0);
    rc = mass_chain(p, u + (size_t)r0 * p->dof, cnt, rhs + (size_t)r0 * p->dof, s);
  }
  if (!rc) {
    const int e = launch_axpy(rhs, b, tau, (long long)total, s);
    if (e) rc = cuda_fail((cudaError_t)e, "heat step right-hand side");
  }
  if (!rc) rc = fem_fft_solve(p, rhs, u_new, nrhs, stream);
  if (rhs != u_new) cudaFreeAsync(rhs, s);
  return rc;
}

int fem_fft_forward_fn(fem_fft_plan p, const double* w, double* c, int64_t nrhs, void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;
  if (!p || !w || !c || nrhs < 0) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = FEM_FFT_OK;
  p->use_fwdc = 1;
  for (int ax = p->N - 1; ax >= 0 && !rc; --ax)
    rc = run_pass(p, MODE_FWD, ax, nrhs, true, ax == p->N - 1 ? (const void*)w : (const void*)c, true, c, true, false,
                  s);
  p->use_fwdc = 0;
  return rc;
}

int fem_fft_inverse(fem_fft_plan p, const double* c, double* w, int64_t nrhs, void* stream) {
  if (p && nrhs == 0) return FEM_FFT_OK;   // nothing to do (pointers may be NULL)
  if (!p || !c || !w || nrhs < 0) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  for (int ax = 0; ax < p->N; ++ax) {
    if ((rc = run_pass(p, MODE_INV, ax, nrhs, true, ax == 0 ? (const void*)c : (const void*)w, true, w, true,
                       false, s)))
      return rc;
  }
  return FEM_FFT_OK;
}

int fem_fft_grad_coeffs(fem_fft_plan p, const double* u, const double* lam, int64_t nrhs, double* h_grad_a,
                        double* h_grad_c, void* stream) {
  if (!p || !u || !lam || !h_grad_a || !h_grad_c || nrhs < 0) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  FEMFFT_CUDA(cudaMemsetAsync(p->d_scalars, 0, 8 * sizeof(double), s), "memset");
  int rc;
  for (int64_t r0 = 0; r0 < nrhs; r0 += p->max_nrhs) {
    const long long cnt = std::min<int64_t>(p->max_nrhs, nrhs - r0);
    if ((rc = grad_chain(p, u + (size_t)r0 * p->dof, lam + (size_t)r0 * p->dof, cnt, p->d_scalars, s))) return rc;
  }
  double h[8];
  FEMFFT_CUDA(cudaMemcpyAsync(h, p->d_scalars, sizeof(h), cudaMemcpyDeviceToHost, s), "dots");
  FEMFFT_CUDA(cudaStreamSynchronize(s), "dots sync");
  for (int i = 0; i < p->N; ++i) h_grad_a[i] = -h[i];
  *h_grad_c = -h[p->N];
  return FEM_FFT_OK;
}

}  // extern "C"

// ------------------------------------------------------------ diagnostics

namespace femfft {
namespace {

__global__ void divide_check_kernel(const double* __restrict__ x, const double* __restrict__ d, double* __restrict__ q,
                                    double* __restrict__ ref, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    q[i] = divide_by(x[i], d[i]);
    ref[i] = x[i] / d[i];
  }
}

}  // namespace
}  // namespace femfft

extern "C" int fem_fft_divide_check(const double* d_x, const double* d_d, double* d_q, double* d_ref, int64_t n,
                                    void* stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_d || !d_q || !d_ref))) return FEM_FFT_ERR_ARG;
  if (n == 0) return FEM_FFT_OK;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  femfft::divide_check_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_x, d_d, d_q, d_ref, n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FEM_FFT_OK : cuda_fail(e, "divide check");
}
