// Batched solves: many problems (uneven N, n, K and right-hand sides) run as
// one dependency-driven launch per element order, all in one CUDA graph.
// Host code; the kernel and the work-list records are in batch_kernel.cuh.
//
// Building a batch: the mixed-precision solve chain of every plan is recorded
// (the launches fem_fft_solve would make), each pencil pass gets the tile
// shape and radix schedule chosen by the autotuner, the chains are cut into
// items and numbered in level order, and one graph is built: per element
// order, a reset of that order's counters followed by its kernel.  The orders
// never wait on each other (every dependency is inside one problem).
//
// Autotuner: for every (n, K, contiguous/strided, pass mode) in the batch it
// times the batch kernel on one-step work lists over a 64 MiB scratch field,
// for pencils per tile W in {1, 2, 4, ..., 32} and FFT values per thread V in
// {4, 8} (powers of two) or {6, 12} (K with a factor 3), and keeps the fastest
// per pencil.  For the fused forward/divide/inverse pass it also times the
// split form (forward with division, then inverse) and keeps the faster.
// Results can be kept in a JSON file keyed by the GPU name.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "batch_kernel.cuh"
#include "plan.h"

using namespace femfft;

namespace {

constexpr const char* kTuneVersion = "femfft-batch-tune-5";

// Relocation tags: the chains are recorded with placeholder addresses
// tag + byte offset for the right-hand sides (b) and solutions (u); every
// solve call with new buffers rewrites them.
constexpr uintptr_t kTagB = uintptr_t(1) << 56;
constexpr uintptr_t kTagU = uintptr_t(2) << 56;
constexpr uintptr_t kTagMask = uintptr_t(0xff) << 56;

const void* kernel_for(int n) {
  if (n >= 1 && n <= 3) return batch_kernel_fn_1(n);
  if (n >= 4 && n <= 6) return batch_kernel_fn_2(n);
  if (n >= 7 && n <= 9) return batch_kernel_fn_3(n);
  return nullptr;
}

struct TuneKey {
  int n, K, strided, mode;
  bool operator<(const TuneKey& o) const {
    return std::tie(n, K, strided, mode) < std::tie(o.n, o.K, o.strided, o.mode);
  }
};
struct TuneVal {
  int W = 0, V = 0;
  int split = 0;                 // fused pass only: run as forward-with-division + inverse
  double us_per_pencil = 0.0;
};

int batch_fail(int code, const std::string& what) {
  set_last_error(what);
  return code;
}

size_t pencil_smem(const PassParams& P) {
  return (size_t)P.g.W * P.pitch * 2 * sizeof(float) + 2 * (size_t)P.ax.K * 2 * sizeof(float);
}

// Dynamic shared memory available to one CTA of the batch kernel of order n
// (kBatchCtasPerSm resident CTAs share an SM).
size_t smem_budget(int n) {
  int dev = 0, optin = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  optin = std::min(optin, per_sm / kBatchCtasPerSm - 1024);
  cudaFuncAttributes fa;
  std::memset(&fa, 0, sizeof(fa));
  const void* fn = kernel_for(n);
  if (!fn || cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
}

// The attribute only grows, so that graphs built for larger tiles stay
// launchable after a later batch or tuning run.
int enable_smem(int n, size_t smem) {
  const int e = ensure_dyn_smem(kernel_for(n), smem);
  if (e) return cuda_fail((cudaError_t)e, "batch kernel shared memory");
  return FEM_FFT_OK;
}

// Largest admissible W for a pass: shared memory, the chunk tasks of the
// sequence build, and (strided pencils) a power of two within the inner run.
int max_tile_w(const PassParams& P, size_t budget) {
  const int K = P.ax.K;
  long long w = kMaxW;
  w = std::min<long long>(w, (long long)kMaxChunkTasks * kBatchThreads / K);
  const int Q = P.ax.n / 2 + 1;
  const size_t per_pen = (size_t)(pencil_pitch_min(K, Q) + kPitchSlack) * 2 * sizeof(float);
  const size_t tables = 2 * (size_t)K * 2 * sizeof(float);
  if (budget <= tables) return 0;
  w = std::min<long long>(w, (long long)((budget - tables) / per_pen));
  if (P.g.inner > 1) {
    const long long lim = std::min<long long>(w, P.g.inner);
    long long p2 = 1;
    while (p2 * 2 <= lim) p2 *= 2;
    w = lim >= 1 ? p2 : 0;
  }
  return (int)std::max<long long>(w, 0);
}

bool set_tile(PassParams& P, int W, int V, size_t budget) {
  const int K = P.ax.K;
  int npass, radix[kMaxRadixPasses];
  if (!fft_schedule_v(K, V, &npass, radix) || K / V > kBatchThreads) return false;
  if (W < 1 || W > max_tile_w(P, budget)) return false;
  if (P.g.inner > 1 && (W & (W - 1))) return false;
  P.V = V;
  P.npass = npass;
  for (int i = 0; i < kMaxRadixPasses; ++i) P.radix[i] = i < npass ? radix[i] : 0;
  set_fft_passes(P);
  set_pass_tiles(P, W);
  P.pitch = tile_pitch(K, P.ax.n / 2 + 1, V, W, P.g.inner > 1, 4);
  return true;
}

// FFT values per thread worth timing for length K.
std::vector<int> v_candidates(int K) {
  std::vector<int> out;
  for (int V : {4, 8, 6, 12}) {
    int np, r[kMaxRadixPasses];
    if (fft_schedule_v(K, V, &np, r) && K / V <= kBatchThreads) out.push_back(V);
  }
  if (out.empty()) out.push_back(K <= 4 ? K : 2);
  return out;
}

BatchArgs make_args(const BatchStage* d_stages, const int* d_items, long long total, unsigned char* d_counters,
                    unsigned long long wait_ns) {
  BatchArgs A;
  A.stages = d_stages;
  A.item_stage = d_items;
  A.total = total;
  A.ticket = reinterpret_cast<unsigned long long*>(d_counters);
  A.status = reinterpret_cast<int*>(d_counters + 8);
  A.where = reinterpret_cast<int*>(d_counters + 12);
  A.done = reinterpret_cast<unsigned*>(d_counters + 16);
  A.wait_ns = wait_ns;
  return A;
}

// Counter block of a work list: ticket (8 bytes), status, where, done[steps].
size_t counter_bytes(size_t steps) { return 16 + sizeof(unsigned) * steps; }

// Numbers the items of steps given in ticket order; prev[i] is the previous
// step of the same problem (-1 for the first).
void number_items(std::vector<BatchStage>& st, const std::vector<int>& prev, std::vector<int>* item_stage,
                  long long* total) {
  long long t = 0;
  for (size_t i = 0; i < st.size(); ++i) {
    st[i].first = t;
    st[i].items = (st[i].units + st[i].units_per_item - 1) / st[i].units_per_item;
    t += st[i].items;
  }
  for (size_t i = 0; i < st.size(); ++i) {
    st[i].dep = prev[i];
    st[i].need = prev[i] >= 0 ? (unsigned)st[prev[i]].items : 0u;
  }
  item_stage->assign((size_t)t, 0);
  for (size_t i = 0; i < st.size(); ++i)
    for (long long k = 0; k < st[i].items; ++k) (*item_stage)[(size_t)(st[i].first + k)] = (int)i;
  *total = t;
}

// ------------------------------------------------------------- autotuner

std::string gpu_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  return prop.name;
}

void load_cache(const char* path, const std::string& gpu, std::map<TuneKey, TuneVal>* out) {
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t r;
  while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, r);
  std::fclose(f);
  if (text.find(std::string("\"version\": \"") + kTuneVersion + "\"") == std::string::npos) return;
  if (text.find("\"gpu\": \"" + gpu + "\"") == std::string::npos) return;
  size_t pos = 0;
  while ((pos = text.find("{\"n\":", pos)) != std::string::npos) {
    TuneKey k;
    TuneVal v;
    if (std::sscanf(text.c_str() + pos,
                    "{\"n\": %d, \"K\": %d, \"strided\": %d, \"mode\": %d, \"W\": %d, \"V\": %d, \"split\": %d, "
                    "\"us_per_pencil\": %lf}",
                    &k.n, &k.K, &k.strided, &k.mode, &v.W, &v.V, &v.split, &v.us_per_pencil) == 8)
      (*out)[k] = v;
    ++pos;
  }
}

void save_cache(const char* path, const std::string& gpu, const std::map<TuneKey, TuneVal>& tab) {
  if (!path || !*path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\"version\": \"%s\", \"gpu\": \"%s\", \"entries\": [\n", kTuneVersion, gpu.c_str());
  size_t i = 0;
  for (const auto& kv : tab) {
    std::fprintf(f,
                 "  {\"n\": %d, \"K\": %d, \"strided\": %d, \"mode\": %d, \"W\": %d, \"V\": %d, \"split\": %d, "
                 "\"us_per_pencil\": %.6g}%s\n",
                 kv.first.n, kv.first.K, kv.first.strided, kv.first.mode, kv.second.W, kv.second.V, kv.second.split,
                 kv.second.us_per_pencil, ++i < tab.size() ? "," : "");
  }
  std::fprintf(f, "]}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}

struct TuneScratch {
  float* field = nullptr;
  size_t floats = size_t(1) << 24;   // 64 MiB
  BatchStage* d_stage = nullptr;
  int* d_items = nullptr;
  size_t max_items = size_t(1) << 20;
  unsigned char* d_counters = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// Times one candidate: a one-step work list (W pencils per tile, V FFT
// values per thread) over the zeroed scratch field.  Returns microseconds
// per pencil, or a negative value if the candidate is not admissible.
double time_candidate(const PassParams& proto, int mode, int W, int V, size_t budget, TuneScratch& ts,
                      cudaStream_t s) {
  BatchStage st;
  std::memset(&st, 0, sizeof(st));
  st.kind = BATCH_PENCIL;
  st.mode = mode;
  st.n = proto.ax.n;
  st.pp = proto;
  if (!set_tile(st.pp, W, V, budget)) return -1.0;
  st.units = st.pp.g.tiles;
  st.units_per_item = 1;
  st.dep = -1;
  st.items = st.units;
  st.first = 0;
  if ((size_t)st.items > ts.max_items) return -1.0;
  const size_t smem = std::max(pencil_smem(st.pp), batch_apply_smem<kMaxOrder>());
  if (enable_smem(st.n, smem)) return -1.0;
  // every ticket maps to step 0 (the item table was zeroed once)
  if (cudaMemcpyAsync(ts.d_stage, &st, sizeof(st), cudaMemcpyHostToDevice, s) != cudaSuccess) return -1.0;
  BatchArgs A = make_args(ts.d_stage, ts.d_items, st.items, ts.d_counters, 2000000000ull);
  void* args[] = {&A};
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    if (cudaMemsetAsync(ts.d_counters, 0, counter_bytes(1), s) != cudaSuccess) return -1.0;
    cudaEventRecord(ts.ev0, s);
    if (cudaLaunchKernel(kernel_for(st.n), dim3((unsigned)st.items), dim3(kBatchThreads), args, smem, s) !=
        cudaSuccess) {
      cudaGetLastError();
      return -1.0;
    }
    cudaEventRecord(ts.ev1, s);
    if (cudaEventSynchronize(ts.ev1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ts.ev0, ts.ev1);
    if (rep > 0) best = std::min(best, ms);
  }
  int status = 0;
  if (cudaMemcpy(&status, ts.d_counters + 8, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      status != FEM_FFT_OK)
    return -1.0;
  const double pencils = (double)proto.g.outer * (double)proto.g.inner;
  return best * 1e3 / pencils;
}

// Best (W, V) of one pass mode for a key; proto carries the key's tables.
// The scratch geometry: contiguous pencils fill the field; strided ones run
// along an axis with 512 pencils side by side.
TuneVal tune_mode(PassParams proto, int mode, int strided, size_t budget, TuneScratch& ts, cudaStream_t s) {
  const int M = proto.g.M;
  proto.in = ts.field;
  proto.out = ts.field;
  proto.in_f64 = proto.out_f64 = proto.accum = 0;
  if (strided) {
    proto.g.inner = 512;
    proto.g.outer = std::max<long long>(1, (long long)(ts.floats / ((size_t)M * 512)));
  } else {
    proto.g.inner = 1;
    proto.g.outer = std::max<long long>(1, (long long)(ts.floats / (size_t)M));
  }
  if (mode == MODE_FUSED || mode == MODE_FWD_DIV) {
    proto.dv.c = 1.0;
    proto.dv.nother = 0;
  }
  TuneVal best;
  best.us_per_pencil = 1e300;
  for (int V : v_candidates(proto.ax.K)) {
    for (int W = 1; W <= kMaxW; W *= 2) {
      const double us = time_candidate(proto, mode, W, V, budget, ts, s);
      if (us > 0 && us < best.us_per_pencil) {
        best.W = W;
        best.V = V;
        best.us_per_pencil = us;
      }
    }
  }
  return best;
}

int tune_keys(const std::map<TuneKey, PassParams>& keys, std::map<TuneKey, TuneVal>* tab, cudaStream_t s) {
  std::vector<TuneKey> todo;
  for (const auto& kv : keys)
    if (!tab->count(kv.first)) todo.push_back(kv.first);
  if (todo.empty()) return FEM_FFT_OK;
  TuneScratch ts;
  int rc = FEM_FFT_OK;
  if (cudaMalloc(&ts.field, ts.floats * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&ts.d_stage, sizeof(BatchStage)) != cudaSuccess ||
      cudaMalloc(&ts.d_items, sizeof(int) * ts.max_items) != cudaSuccess ||
      cudaMalloc(&ts.d_counters, 64) != cudaSuccess) {
    cudaGetLastError();
    rc = batch_fail(FEM_FFT_ERR_OOM, "autotuner scratch");
  }
  if (!rc) {
    cudaEventCreate(&ts.ev0);
    cudaEventCreate(&ts.ev1);
    if (cudaMemsetAsync(ts.field, 0, ts.floats * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(ts.d_items, 0, sizeof(int) * ts.max_items, s) != cudaSuccess)
      rc = batch_fail(FEM_FFT_ERR_CUDA, "autotuner scratch");
  }
  for (size_t i = 0; i < todo.size() && !rc; ++i) {
    const TuneKey& k = todo[i];
    const PassParams& proto = keys.at(k);
    const size_t budget = smem_budget(k.n);
    TuneVal v = tune_mode(proto, k.mode, k.strided, budget, ts, s);
    if (v.W == 0) {
      rc = batch_fail(FEM_FFT_ERR_ARG, "autotuner: no admissible tile");
      break;
    }
    if (k.mode == MODE_FUSED) {
      // the split form: forward with division, then the inverse pass
      TuneVal a = tune_mode(proto, MODE_FWD_DIV, k.strided, budget, ts, s);
      TuneKey kinv{k.n, k.K, k.strided, MODE_INV};
      TuneVal bv = tab->count(kinv) ? (*tab)[kinv] : tune_mode(proto, MODE_INV, k.strided, budget, ts, s);
      if (a.W && bv.W) {
        (*tab)[TuneKey{k.n, k.K, k.strided, MODE_FWD_DIV}] = a;
        (*tab)[kinv] = bv;
        if (a.us_per_pencil + bv.us_per_pencil < v.us_per_pencil) v.split = 1;
      }
    }
    (*tab)[k] = v;
  }
  if (ts.ev0) cudaEventDestroy(ts.ev0);
  if (ts.ev1) cudaEventDestroy(ts.ev1);
  cudaFree(ts.field);
  cudaFree(ts.d_stage);
  cudaFree(ts.d_items);
  cudaFree(ts.d_counters);
  cudaGetLastError();
  return rc;
}

void relocate(BatchStage& st, const double* b, double* u) {
  auto fix = [&](const void* p) -> void* {
    const uintptr_t v = reinterpret_cast<uintptr_t>(p);
    if ((v & kTagMask) == kTagB) return (void*)(reinterpret_cast<const char*>(b) + (v - kTagB));
    if ((v & kTagMask) == kTagU) return (void*)(reinterpret_cast<char*>(u) + (v - kTagU));
    return const_cast<void*>(p);
  };
  if (st.kind == BATCH_PENCIL) {
    st.pp.in = fix(st.pp.in);
    st.pp.out = fix(st.pp.out);
  } else {
    for (int i = 0; i < kApplyMaxIn; ++i) st.ap.in[i] = (const double*)fix(st.ap.in[i]);
    for (int i = 0; i < kApplyMaxOut; ++i) st.ap.out[i] = (double*)fix(st.ap.out[i]);
    st.ap.base = (const double*)fix(st.ap.base);
    st.ap.addend = (const double*)fix(st.ap.addend);
  }
}

}  // namespace

// One element order's share of a batch: its steps in ticket order, items and
// counters, launched as one kernel.
struct BatchGroup {
  int n = 0;
  std::vector<BatchStage> stages;
  std::vector<int> item_stage;
  long long total_items = 0;
  size_t smem = 0;
  BatchStage* d_stages = nullptr;
  int* d_item_stage = nullptr;
  unsigned char* d_counters = nullptr;
  size_t counters_bytes = 0;
};

struct fem_fft_batch_s {
  int nprob = 0, steps = 2;
  std::vector<int64_t> nrhs, offset;   // offset: first float64 of problem p in the packed buffers
  int64_t total_len = 0;
  std::vector<BatchGroup> groups;
  int hold_group = -1, hold_step = -1; // a step whose dependency target is made unreachable (tests)
  const double* cur_b = nullptr;
  double* cur_u = nullptr;
  bool uploaded = false;
  unsigned long long wait_ns = 2000000000ull;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<std::pair<TuneKey, TuneVal>> tune_used;
  // stream mode (fem_fft_batch_set_mode): every problem solved by its own
  // plan (fem_fft_solve, the plan's fastest kernels) on one of nstreams
  // streams, problems assigned largest first to the least loaded stream
  std::vector<fem_fft_plan> plans;
  std::vector<double> work;
  int mode = FEM_FFT_BATCH_GRAPH;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  std::vector<int> order, stream_of;
  bool graph_ok = true;   // false: some plan has different orders on its axes (stream mode only)
};

namespace {

void drop_graph(fem_fft_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void drop_streams(fem_fft_batch b) {
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  b->streams.clear();
  b->join.clear();
  b->fork = nullptr;
}

void free_batch(fem_fft_batch b) {
  if (!b) return;
  drop_graph(b);
  drop_streams(b);
  for (auto& g : b->groups) {
    cudaFree(g.d_stages);
    cudaFree(g.d_item_stage);
    cudaFree(g.d_counters);
  }
  delete b;
}

int build_graph(fem_fft_batch b) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch graph");
  for (auto& gr : b->groups) {
    if (gr.total_items == 0) continue;
    cudaMemsetParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.dst = gr.d_counters;
    mp.value = 0;
    mp.elementSize = 1;
    mp.width = gr.counters_bytes;
    mp.height = 1;
    mp.pitch = gr.counters_bytes;
    cudaGraphNode_t nmem = nullptr, nker = nullptr;
    BatchArgs A = make_args(gr.d_stages, gr.d_item_stage, gr.total_items, gr.d_counters, b->wait_ns);
    void* args[] = {&A};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = const_cast<void*>(kernel_for(gr.n));
    kp.gridDim = dim3((unsigned)gr.total_items);
    kp.blockDim = dim3(kBatchThreads);
    kp.sharedMemBytes = (unsigned)gr.smem;
    kp.kernelParams = args;
    e = cudaGraphAddMemsetNode(&nmem, g, nullptr, 0, &mp);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&nker, g, &nmem, 1, &kp);
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return cuda_fail(e, "batch graph build");
  }
  b->graph = g;
  b->exec = ex;
  return FEM_FFT_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" {

int fem_fft_batch_order(int nprob, const int* nsteps, const double* work, int* h_prob, int* h_step) {
  if (nprob < 0 || (nprob > 0 && (!nsteps || !h_prob || !h_step))) return FEM_FFT_ERR_ARG;
  std::vector<int> order(nprob);
  for (int p = 0; p < nprob; ++p) order[p] = p;
  if (work) std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  int maxs = 0;
  for (int p = 0; p < nprob; ++p) {
    if (nsteps[p] < 0) return FEM_FFT_ERR_ARG;
    maxs = std::max(maxs, nsteps[p]);
  }
  int k = 0;
  for (int l = 0; l < maxs; ++l)
    for (int p : order)
      if (l < nsteps[p]) {
        h_prob[k] = p;
        h_step[k] = l;
        ++k;
      }
  return k;
}

int fem_fft_batch_create(fem_fft_batch* out, const fem_fft_plan* plans, int nprob, const int64_t* h_nrhs,
                         int steps, const char* tune_cache, int tune, void* stream) {
  if (!out) return FEM_FFT_ERR_ARG;
  *out = nullptr;
  if (nprob < 1 || !plans || !h_nrhs || steps < 0 || steps > 16)
    return batch_fail(FEM_FFT_ERR_ARG, "batch: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  fem_fft_batch b = new (std::nothrow) fem_fft_batch_s();
  if (!b) return FEM_FFT_ERR_OOM;
  b->nprob = nprob;
  b->steps = steps;
  // A plan with different orders on its axes would span launches of the
  // batched kernel (one per element order): such a batch runs in stream mode
  // only (no recording, no graph).
  bool uniform_all = true;
  for (int p = 0; p < nprob; ++p) {
    fem_fft_plan pl = plans[p];
    for (int i = 1; pl && i < pl->N; ++i) uniform_all = uniform_all && pl->nax[i] == pl->nax[0];
  }
  b->graph_ok = uniform_all;
  // 1. record every problem's solve chain with placeholder field addresses
  int64_t off = 0;
  std::vector<std::vector<RecordedOp>> chains(nprob);
  std::vector<double> work(nprob);
  for (int p = 0; p < nprob; ++p) {
    fem_fft_plan pl = plans[p];
    if (!pl || pl->precision != FEM_FFT_MIXED || h_nrhs[p] < 1 || h_nrhs[p] > pl->max_nrhs) {
      free_batch(b);
      return batch_fail(FEM_FFT_ERR_ARG, "batch: every plan must be mixed precision with nrhs <= max_nrhs");
    }
    for (int q = 0; q < p; ++q)
      if (plans[q] == pl) {
        free_batch(b);
        return batch_fail(FEM_FFT_ERR_ARG, "batch: a plan appears twice (its workspace would be shared)");
      }
    b->nrhs.push_back(h_nrhs[p]);
    b->offset.push_back(off);
    const double* tb = reinterpret_cast<const double*>(kTagB + (uintptr_t)off * sizeof(double));
    double* tu = reinterpret_cast<double*>(kTagU + (uintptr_t)off * sizeof(double));
    int rc = uniform_all ? record_mixed_solve(pl, tb, tu, h_nrhs[p], steps, &chains[p]) : FEM_FFT_OK;
    if (rc) {
      free_batch(b);
      return batch_fail(rc, "batch: recording a solve chain failed");
    }
    off += h_nrhs[p] * pl->dof;
    work[p] = (double)h_nrhs[p] * (double)pl->dof;
  }
  b->total_len = off;
  b->plans.assign(plans, plans + nprob);
  b->work = work;
  if (!uniform_all) {
    const int rc = fem_fft_batch_set_mode(b, FEM_FFT_BATCH_STREAMS, 4);
    if (rc) {
      free_batch(b);
      return rc;
    }
    *out = b;
    return FEM_FFT_OK;
  }
  // 2. tile shapes and radix schedules
  std::map<TuneKey, PassParams> keys;
  for (auto& ch : chains)
    for (auto& op : ch)
      if (op.kind == 0) {
        TuneKey k{op.pp.ax.n, op.pp.ax.K, op.pp.g.inner > 1 ? 1 : 0, op.mode};
        if (!keys.count(k)) keys[k] = op.pp;
      }
  std::map<TuneKey, TuneVal> tab;
  const std::string gpu = gpu_name();
  load_cache(tune_cache, gpu, &tab);
  if (tune) {
    int rc = tune_keys(keys, &tab, s);
    if (rc) {
      free_batch(b);
      return rc;
    }
    save_cache(tune_cache, gpu, tab);
  }
  for (const auto& kv : keys) {
    auto it = tab.find(kv.first);
    if (it != tab.end()) b->tune_used.push_back(*it);
  }
  // 3. per problem: the chain as batch steps (tuned tiles; fused passes split
  //    where the tuner found that faster)
  std::vector<std::vector<BatchStage>> psteps(nprob);
  for (int p = 0; p < nprob; ++p) {
    for (const RecordedOp& op : chains[p]) {
      BatchStage st;
      std::memset(&st, 0, sizeof(st));
      if (op.kind == 0) {
        const int n = op.pp.ax.n, K = op.pp.ax.K;
        const size_t budget = smem_budget(n);
        const int strided = op.pp.g.inner > 1 ? 1 : 0;
        auto tiled = [&](int mode, PassParams P, BatchStage* o) {
          bool ok = false;
          auto it = tab.find(TuneKey{n, K, strided, mode});
          if (it != tab.end()) {
            const int W = std::min(it->second.W, max_tile_w(P, budget));
            ok = W >= 1 && set_tile(P, W, it->second.V, budget);
          }
          if (!ok) {   // the stand-alone pass's schedule, W clipped to the budget
            const int W = std::min(op.pp.g.W, max_tile_w(P, budget));
            ok = W >= 1 && set_tile(P, W, op.pp.V, budget);
          }
          if (!ok) return false;
          std::memset(o, 0, sizeof(*o));
          o->kind = BATCH_PENCIL;
          o->mode = mode;
          o->n = n;
          o->pp = P;
          o->units = P.g.tiles;
          o->units_per_item = 1;
          return true;
        };
        auto itf = tab.find(TuneKey{n, K, strided, MODE_FUSED});
        const bool split = op.mode == MODE_FUSED && !op.pp.out_f64 && !op.pp.accum && itf != tab.end() &&
                           itf->second.split;
        bool ok;
        if (split) {
          BatchStage a, c;
          PassParams pinv = op.pp;
          pinv.in = op.pp.out;
          pinv.in_f64 = op.pp.out_f64;
          ok = tiled(MODE_FWD_DIV, op.pp, &a) && tiled(MODE_INV, pinv, &c);
          if (ok) {
            psteps[p].push_back(a);
            psteps[p].push_back(c);
          }
        } else {
          ok = tiled(op.mode, op.pp, &st);
          if (ok) psteps[p].push_back(st);
        }
        if (!ok) {
          free_batch(b);
          return batch_fail(FEM_FFT_ERR_ARG, "batch: a pencil does not fit the batch kernel's shared memory");
        }
      } else if (op.kind == 2) {
        // algorithm (b): condensation, vertex solve, back substitution
        if (op.mode != 0) {
          free_batch(b);
          return batch_fail(FEM_FFT_ERR_ARG, "batch: band solves run in float32 only");
        }
        const BandParams& B = op.bp;
        const int TW = band_tw(B.inner);
        const long long eblocks = band_elem_blocks(B, TW);
        for (int phase = 0; phase < 3; ++phase) {
          BatchStage bs;
          std::memset(&bs, 0, sizeof(bs));
          bs.kind = BATCH_BAND;
          bs.mode = phase;
          bs.n = B.n;
          bs.TW = TW;
          bs.bp = B;
          bs.units = phase == 1 ? band_vertex_blocks(B) : eblocks;
          bs.units_per_item =
              phase == 1 ? 1 : (int)std::max<long long>(1, kItemDof / ((long long)kBandThreads * B.n));
          if (phase == 2 && B.n == 1) continue;   // no interiors to recover
          psteps[p].push_back(bs);
        }
      } else {
        if (op.ap.nout > 2 || op.ap.dotv || op.ap.norms || (op.ap.df && !apply_df_form_ok(op.ap))) {
          free_batch(b);
          return batch_fail(FEM_FFT_ERR_ARG, "batch: unsupported apply form");
        }
        st.kind = BATCH_APPLY;
        st.ap = op.ap;
        st.mode = op.ap.df ? apply_df_nacc(op.ap) : op.ap.nout;
        st.n = op.ap.n;
        const int TW = apply_tile_w(op.ap.inner, op.ap.outer, op.ap.K, kBatchThreads);
        st.TW = TW;
        st.units = apply_tile_blocks(op.ap.inner, op.ap.outer, op.ap.K, TW, kBatchThreads);
        st.units_per_item = (int)std::max<long long>(1, kItemDof / ((long long)kBatchThreads * op.ap.n));
        if (op.ap.df) {
          int nin = 0;
          for (int i = 0; i < kApplyMaxIn; ++i) nin += op.ap.in[i] != nullptr;
          st.tile_smem = (int)apply_df_tile_bytes(op.ap.n, TW, kBatchThreads, nin);   // staged input tiles
          // one tile per output where the CTA has room, so that the outputs of
          // narrow blocks leave coalesced (as in the stand-alone launch)
          const int cap = std::max(nin, op.ap.nout);
          const size_t with_out = apply_df_tile_bytes(op.ap.n, TW, kBatchThreads, cap);
          if (cap > nin && batch_apply_smem<kMaxOrder>() + with_out <= smem_budget(op.ap.n)) {
            st.tile_smem = (int)with_out;
            st.ap.tile_cap = cap;
          }
        }
        psteps[p].push_back(st);
      }
    }
  }
  // 4. per element order: steps in level order, items, device arrays
  for (int n = 1; n <= kMaxOrder; ++n) {
    std::vector<int> probs;
    for (int p = 0; p < nprob; ++p)
      if (plans[p]->n == n) probs.push_back(p);
    if (probs.empty()) continue;
    BatchGroup g;
    g.n = n;
    std::vector<int> nst(probs.size());
    std::vector<double> w(probs.size());
    size_t total = 0;
    for (size_t i = 0; i < probs.size(); ++i) {
      nst[i] = (int)psteps[probs[i]].size();
      w[i] = work[probs[i]];
      total += nst[i];
    }
    std::vector<int> oprob(total), ostep(total);
    fem_fft_batch_order((int)probs.size(), nst.data(), w.data(), oprob.data(), ostep.data());
    std::vector<int> prev(total, -1), last(probs.size(), -1);
    g.smem = batch_apply_smem<kMaxOrder>();
    for (size_t i = 0; i < total; ++i) {
      const BatchStage& st = psteps[probs[oprob[i]]][ostep[i]];
      if (st.kind == BATCH_PENCIL) g.smem = std::max(g.smem, pencil_smem(st.pp));
      else if (st.kind == BATCH_BAND) g.smem = std::max(g.smem, sizeof(BandParams));
      else g.smem = std::max(g.smem, batch_apply_smem<kMaxOrder>() + (size_t)st.tile_smem);
      g.stages.push_back(st);
      prev[i] = last[oprob[i]];
      last[oprob[i]] = (int)i;
    }
    number_items(g.stages, prev, &g.item_stage, &g.total_items);
    if (g.total_items >= (1ll << 31) - 1) {
      free_batch(b);
      return batch_fail(FEM_FFT_ERR_ARG, "batch: too many work items");
    }
    int rc = enable_smem(n, g.smem);
    if (rc) {
      free_batch(b);
      return rc;
    }
    g.counters_bytes = counter_bytes(g.stages.size());
    b->groups.push_back(g);
    BatchGroup& G = b->groups.back();
    if (cudaMalloc(&G.d_stages, sizeof(BatchStage) * G.stages.size()) != cudaSuccess ||
        cudaMalloc(&G.d_item_stage, sizeof(int) * G.item_stage.size()) != cudaSuccess ||
        cudaMalloc(&G.d_counters, G.counters_bytes) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return batch_fail(FEM_FFT_ERR_OOM, "batch: device arrays");
    }
    if (cudaMemcpyAsync(G.d_item_stage, G.item_stage.data(), sizeof(int) * G.item_stage.size(),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(G.d_counters, 0, G.counters_bytes, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return batch_fail(FEM_FFT_ERR_CUDA, "batch: upload");
    }
  }
  *out = b;
  return FEM_FFT_OK;
}

int fem_fft_batch_destroy(fem_fft_batch b) {
  if (!b) return FEM_FFT_ERR_ARG;
  cudaDeviceSynchronize();
  free_batch(b);
  return FEM_FFT_OK;
}

int fem_fft_batch_layout(fem_fft_batch b, int64_t* h_offsets, int64_t* total_len, int64_t* n_steps,
                         int64_t* n_items) {
  if (!b) return FEM_FFT_ERR_ARG;
  if (h_offsets)
    for (int p = 0; p < b->nprob; ++p) h_offsets[p] = b->offset[p];
  if (total_len) *total_len = b->total_len;
  int64_t ns = 0, ni = 0;
  for (const auto& g : b->groups) {
    ns += (int64_t)g.stages.size();
    ni += g.total_items;
  }
  if (n_steps) *n_steps = ns;
  if (n_items) *n_items = ni;
  return FEM_FFT_OK;
}

int fem_fft_batch_tuning(fem_fft_batch b, int max_entries, int* h_entries, double* h_us) {
  if (!b || max_entries < 0) return FEM_FFT_ERR_ARG;
  const int cnt = (int)b->tune_used.size();
  for (int i = 0; i < std::min(cnt, max_entries); ++i) {
    const auto& e = b->tune_used[i];
    if (h_entries) {
      int* r = h_entries + 7 * i;
      r[0] = e.first.n;
      r[1] = e.first.K;
      r[2] = e.first.strided;
      r[3] = e.first.mode;
      r[4] = e.second.W;
      r[5] = e.second.V;
      r[6] = e.second.split;
    }
    if (h_us) h_us[i] = e.second.us_per_pencil;
  }
  return cnt;
}

int fem_fft_batch_set_wait_limit(fem_fft_batch b, double seconds) {
  if (!b || !(seconds > 0.0) || seconds > 600.0) return FEM_FFT_ERR_ARG;
  b->wait_ns = (unsigned long long)(seconds * 1e9);
  drop_graph(b);
  return FEM_FFT_OK;
}

int fem_fft_batch_hold_step(fem_fft_batch b, int64_t step) {
  if (!b || step < -1) return FEM_FFT_ERR_ARG;
  if (step == -1) {
    b->hold_group = b->hold_step = -1;
    b->uploaded = false;
    return FEM_FFT_OK;
  }
  int64_t k = step;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const int64_t ns = (int64_t)b->groups[gi].stages.size();
    if (k < ns) {
      if (b->groups[gi].stages[k].dep < 0) return FEM_FFT_ERR_ARG;
      b->hold_group = (int)gi;
      b->hold_step = (int)k;
      b->uploaded = false;
      return FEM_FFT_OK;
    }
    k -= ns;
  }
  return FEM_FFT_ERR_ARG;
}

int fem_fft_batch_set_mode(fem_fft_batch b, int mode, int nstreams) {
  if (!b || (mode != FEM_FFT_BATCH_GRAPH && mode != FEM_FFT_BATCH_STREAMS)) return FEM_FFT_ERR_ARG;
  if (mode == FEM_FFT_BATCH_GRAPH && !b->graph_ok)
    return batch_fail(FEM_FFT_ERR_ARG, "batch: plans with per-axis orders run in stream mode only");
  if (mode == FEM_FFT_BATCH_STREAMS && (nstreams < 1 || nstreams > 64)) return FEM_FFT_ERR_ARG;
  cudaDeviceSynchronize();   // no solve of either mode may still use the streams
  drop_streams(b);
  b->mode = mode;
  if (mode == FEM_FFT_BATCH_GRAPH) return FEM_FFT_OK;
  b->streams.assign(nstreams, nullptr);
  b->join.assign(nstreams, nullptr);
  for (int i = 0; i < nstreams; ++i)
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      drop_streams(b);
      b->mode = FEM_FFT_BATCH_GRAPH;
      return batch_fail(FEM_FFT_ERR_CUDA, "batch: stream mode set-up");
    }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    drop_streams(b);
    b->mode = FEM_FFT_BATCH_GRAPH;
    return batch_fail(FEM_FFT_ERR_CUDA, "batch: stream mode set-up");
  }
  // largest problems first, each to the stream with the least work so far
  b->order.resize(b->nprob);
  for (int p = 0; p < b->nprob; ++p) b->order[p] = p;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return b->work[x] > b->work[y]; });
  std::vector<double> load(nstreams, 0.0);
  b->stream_of.assign(b->nprob, 0);
  for (int p : b->order) {
    const int i = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->stream_of[p] = i;
    load[i] += b->work[p];
  }
  return FEM_FFT_OK;
}

namespace {

// Stream mode: fork the batch streams from s, solve every problem with its
// plan (refinement steps: the batch's), join back into s.
int solve_streams(fem_fft_batch b, const double* d_b, double* d_u, cudaStream_t s) {
  if (cudaEventRecord(b->fork, s) != cudaSuccess) return cuda_fail(cudaGetLastError(), "batch: fork");
  for (cudaStream_t st : b->streams)
    if (cudaStreamWaitEvent(st, b->fork, 0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "batch: fork");
  int rc = FEM_FFT_OK;
  for (int p : b->order) {
    fem_fft_plan pl = b->plans[p];
    const double rtol = pl->rtol;
    const int iters = pl->max_iter;
    pl->rtol = 0.0;
    pl->max_iter = b->steps;
    rc = fem_fft_solve(pl, d_b + b->offset[p], d_u + b->offset[p], b->nrhs[p], b->streams[b->stream_of[p]]);
    pl->rtol = rtol;
    pl->max_iter = iters;
    if (rc) break;
  }
  for (size_t i = 0; i < b->streams.size(); ++i) {
    if (cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess || cudaStreamWaitEvent(s, b->join[i], 0) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "batch: join");
  }
  return rc;
}

}  // namespace

int fem_fft_batch_solve(fem_fft_batch b, const double* d_b, double* d_u, void* stream) {
  if (!b || !d_b || !d_u) return FEM_FFT_ERR_ARG;
  if ((const void*)d_b == (const void*)d_u) return batch_fail(FEM_FFT_ERR_ARG, "batch: b and u must differ");
  cudaStream_t s = (cudaStream_t)stream;
  if (b->mode == FEM_FFT_BATCH_STREAMS) return solve_streams(b, d_b, d_u, s);
  if (!b->uploaded || d_b != b->cur_b || d_u != b->cur_u) {
    // the previous solve may still read the step tables
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return batch_fail(FEM_FFT_ERR_CUDA, "batch: synchronize");
    }
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
      BatchGroup& g = b->groups[gi];
      std::vector<BatchStage> st = g.stages;
      for (auto& x : st) relocate(x, d_b, d_u);
      if ((int)gi == b->hold_group) st[b->hold_step].need += 1;   // a count its predecessor never reaches
      if (cudaMemcpy(g.d_stages, st.data(), sizeof(BatchStage) * st.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return batch_fail(FEM_FFT_ERR_CUDA, "batch: step table upload");
      }
    }
    b->cur_b = d_b;
    b->cur_u = d_u;
    b->uploaded = true;
  }
  if (!b->exec) {
    int rc = build_graph(b);
    if (rc) return rc;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
  return FEM_FFT_OK;
}

int fem_fft_batch_status(fem_fft_batch b, void* stream, int* h_status, int64_t* h_step) {
  if (!b) return FEM_FFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return batch_fail(FEM_FFT_ERR_CUDA, "batch: synchronize");
  }
  int status = FEM_FFT_OK;
  int64_t where = -1, base = 0;
  for (const auto& g : b->groups) {
    int v[2] = {0, -1};
    if (cudaMemcpy(v, g.d_counters + 8, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return batch_fail(FEM_FFT_ERR_CUDA, "batch: status read");
    }
    if (v[0] != FEM_FFT_OK && status == FEM_FFT_OK) {
      status = v[0];
      where = base + v[1];
    }
    base += (int64_t)g.stages.size();
  }
  if (h_status) *h_status = status;
  if (h_step) *h_step = where;
  return status;
}

}  // extern "C"
