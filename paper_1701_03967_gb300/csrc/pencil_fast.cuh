// Register-radix pencil passes: the direct FC_n-transform, the inverse
// F_n-transform and the fused forward / spectral-divide / inverse pass along
// one axis, for power-of-two element counts 16 <= K <= 1024.
//
// Method (Zlotnik & Zlotnik, arXiv:1701.03967, Section 3, Theorem 2 and
// Section 4, algorithm (a)): the same half-sample DCT-II / DCT-III
// formulation as pencil.cuh (whose header derives it): per pencil, the node
// sum/difference and the even/odd interior combinations form Q = n/2 + 1
// packed complex sequences of length K; one complex FFT per sequence gives
// every half-sample sine and cosine sum; per frequency k the n x 2Q maps of
// Theorem 2 give the FC_n coefficients (item 2) and, transposed, the inputs
// of the inverse F_n-transform (item 1).
//
// What differs from pencil.cuh is the mapping onto the GPU:
//  * FFT: Stockham passes of radix R in {2, 4, 8, 16, 32} evaluated in
//    registers (each thread holds V = 16 or 32 values and runs V / R
//    butterflies per pass), so K = 1024 takes two passes (32 x 32) and one
//    exchange through shared memory.  A sequence belongs to K / V <= 32
//    threads of one warp: passes synchronise with __syncwarp only.  The
//    intermediate buffer of the exchange is XOR-swizzled in its element
//    index (e ^ ((e >> s) & m)), which makes the strided writes of the first
//    pass and the reads of the second conflict-free; the twiddles between
//    the passes are applied as the first pass stores (four-step form), read
//    from a table laid out so that the lanes of a warp read contiguously.
//  * Maps: one thread per (frequency pair (k, K-k), pencil).  It reads both
//    chunks once, applies the DCT post-twiddle, the forward map, the
//    division and the inverse map and the pre-twiddle in registers, and
//    writes both chunks once (the shared-memory stage pencil.cuh spends in
//    four sweeps).  The forward and inverse maps share one table: the
//    forward map of frequency k is F_k[l][j] = c_j G_k[j][l] / ||s_k^(l)||^2
//    with G_k the inverse map (c_j = 1/2 on the node slots, 1 elsewhere), so
//    G (laid out [j][l][k], frequencies contiguous) and the reciprocal norms
//    are all that is read.
//  * Chunks are Qp = Q rounded up to an odd count of complex values, so that
//    consecutive elements fall in distinct banks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pencil.cuh"

namespace femfft {

// Launch shape of the register-radix kernels per (V, mode), compiled into
// their launch bounds and used by the host plan:
//   V = 32 forward and inverse passes: 160 threads (five warps), three CTAs
//     per SM, 128 registers per thread (ptxas spills 448 B per thread; at
//     two CTAs of 320 threads, 96 registers, it spilled 1.3 KB and the
//     spill traffic doubled the DRAM bytes of a launch).  Measured per 2D
//     n = 9 K = 1024 launch: forward 0.63 -> 0.57 ms, inverse 0.79 -> 0.70 ms
//     against that shape (and 1.04 / 0.99 ms with one CTA of 168 registers);
//   V = 32 fused pass (strided pencils): 320 threads, one CTA per SM (168
//     registers): 0.85 ms against 0.91 ms for two CTAs of 160 threads;
//   V = 16: 512 threads, one CTA per SM.
template <int V, int MODE>
__host__ __device__ constexpr int fast_threads() { return V == 32 ? (MODE == 2 ? 320 : 160) : 512; }
template <int V, int MODE>
__host__ __device__ constexpr int fast_min_blocks() { return (V == 32 && MODE != 2) ? 3 : 1; }
// the same at run time (host)
inline int fast_threads_rt(int V, int mode) {
  if (V == 32) return mode == 2 ? fast_threads<32, 2>() : fast_threads<32, 0>();
  return fast_threads<16, 0>();
}
inline int fast_ctas_rt(int V, int mode) {
  if (V == 32) return mode == 2 ? fast_min_blocks<32, 2>() : fast_min_blocks<32, 0>();
  return fast_min_blocks<16, 0>();
}
// chunks per thread of the sequence build (W K <= kFastChunkTasks threads)
constexpr int kFastChunkTasks = 16;

struct FastParams {
  const void* in;
  void* out;
  PassGeom g;
  int K, Qp;           // elements per axis, complex slots per chunk (odd)
  int pitch;           // complex values per pencil in shared memory
  int V, Tn;           // FFT values per thread, threads per sequence (K / V)
  int npass;
  int radix[kFastMaxPass];
  int lprod[kFastMaxPass];   // product of the earlier radices
  int twofs[kFastMaxPass];   // (unused: one four-step table)
  int swz[kFastMaxPass];     // swizzle shift of the buffer written by pass s (0: none)
  int seq_order;             // 0: sequence s = pencil * Q + q; 1: s = q * W + pencil
  const void* tw2;     // T2 [R0][K / R0]: four-step twiddles exp(-2 pi i r i / K)
  const void* rot;     // T2 [K]: exp(-i pi k / (2K))
  const void* gmap;    // T [2Q][n][K]: inverse map G_k[j][l]
  const void* invn;    // T [n][K]: 1 / ||s_k^(l)||_C^2 (k = 0: 1/K for the bubble modes)
  const void* muk;     // T [n][K]: a s lambda of mode (k, l) (k = 0: the bubble modes)
  DivideDev dv;
  int in_f64, out_f64, accum;
  int ahead;           // L2 prefetch distance in tiles (the resident CTAs of the grid; 0: none)
  int* nonfinite;      // if set: raised (atomicOr 1) when a float64 input value is NaN or Inf
};

// ------------------------------------------------------------ DFT kernels

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// cos(2 pi m / 32) for m = 0..8 (first octant), written out to 36 digits
__host__ __device__ constexpr double oct32(int m) {
  return m == 0   ? 1.0
         : m == 1 ? 0.980785280403230449126182236134239037
         : m == 2 ? 0.923879532511286756128183189396788287
         : m == 3 ? 0.831469612302545237078788377617905757
         : m == 4 ? 0.707106781186547524400844362104849039
         : m == 5 ? 0.555570233019602224742830813948532874
         : m == 6 ? 0.382683432365089771728459984030398867
         : m == 7 ? 0.195090322016128267848284868477022241
                  : 0.0;
}
// cos(2 pi m / 32) for any m, by the symmetries of the cosine
__host__ __device__ constexpr double cos32(int m) {
  return (m & 31) <= 8    ? oct32(m & 31)
         : (m & 31) <= 16 ? -oct32(16 - (m & 31))
         : (m & 31) <= 24 ? -oct32((m & 31) - 16)
                          : oct32(32 - (m & 31));
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }

// x * exp(-2 pi i m / R) for a compile-time angle (R divides 32); the
// multiples of pi/4 cost no multiplication or one.
template <typename T, int R, int M>
__device__ __forceinline__ cpx<T> twc(cpx<T> x) {
  constexpr int m = ((M % R) + R) % R;
  constexpr int m32 = m * (32 / R);
  if constexpr (m == 0) {
    return x;
  } else if constexpr (m32 % 8 == 0) {
    constexpr int quarter = m32 / 8;   // exp(-i pi/2 quarter)
    if constexpr (quarter == 1) return {x.im, -x.re};
    else if constexpr (quarter == 2) return {-x.re, -x.im};
    else return {-x.im, x.re};
  } else if constexpr (m32 % 4 == 0) {
    constexpr T c = T(cos32(m32)), s = T(sin32(m32));   // |c| = |s| = sqrt(1/2)
    return {c * x.re + s * x.im, c * x.im - s * x.re};
  } else {
    constexpr T c = T(cos32(m32)), s = T(sin32(m32));
    return {fmaT(c, x.re, s * x.im), fmaT(c, x.im, -s * x.re)};
  }
}

template <typename T, int R>
struct Dft;
template <typename T>
struct Dft<T, 1> {
  __device__ __forceinline__ static void run(cpx<T>*) {}
};
template <typename T>
struct Dft<T, 2> {
  __device__ __forceinline__ static void run(cpx<T>* u) { dft2(u); }
};
template <typename T>
struct Dft<T, 4> {
  __device__ __forceinline__ static void run(cpx<T>* u) { dft4(u); }
};
template <typename T>
struct Dft<T, 8> {
  __device__ __forceinline__ static void run(cpx<T>* u) { dft8(u); }
};

// Cooley-Tukey split R = R1 * R2 in registers:
//   X[k1 + R1 k2] = sum_j2 w_R^(j2 k1) w_R2^(j2 k2) sum_j1 x[j2 + R2 j1] w_R1^(j1 k1)
template <typename T, int R1, int R2>
struct DftSplit {
  template <int J2>
  __device__ __forceinline__ static void inner(const cpx<T>* u, cpx<T>* a) {
    cpx<T> t[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1) t[j1] = u[J2 + R2 * j1];
    Dft<T, R1>::run(t);
    twid_row<J2, 0>(t, a);
  }
  template <int J2, int K1>
  __device__ __forceinline__ static void twid_row(const cpx<T>* t, cpx<T>* a) {
    if constexpr (K1 < R1) {
      a[K1 * R2 + J2] = twc<T, R1 * R2, J2 * K1>(t[K1]);
      twid_row<J2, K1 + 1>(t, a);
    }
  }
  template <int J2>
  __device__ __forceinline__ static void all_inner(const cpx<T>* u, cpx<T>* a) {
    if constexpr (J2 < R2) {
      inner<J2>(u, a);
      all_inner<J2 + 1>(u, a);
    }
  }
  __device__ __forceinline__ static void run(cpx<T>* u) {
    cpx<T> a[R1 * R2];
    all_inner<0>(u, a);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      cpx<T> t[R2];
#pragma unroll
      for (int j2 = 0; j2 < R2; ++j2) t[j2] = a[k1 * R2 + j2];
      Dft<T, R2>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) u[k1 + R1 * k2] = t[k2];
    }
  }
};
template <typename T>
struct Dft<T, 16> {
  __device__ __forceinline__ static void run(cpx<T>* u) { DftSplit<T, 4, 4>::run(u); }
};
template <typename T>
struct Dft<T, 32> {
  __device__ __forceinline__ static void run(cpx<T>* u) { DftSplit<T, 8, 4>::run(u); }
};

// ------------------------------------------------------------- FFT engine

// XOR swizzle of an element index: bits [0, min(sh, 4)) flipped by the bits
// above them (a bijection within every aligned block of 16, so within [0, K))
__host__ __device__ __forceinline__ int swz_pos(int e, int sh) {
  return sh ? (e ^ ((e >> sh) & ((1 << (sh < 4 ? sh : 4)) - 1))) : e;
}

// One Stockham pass of radix R over one sequence (element e at base[pos(e) Qp]).
// Butterfly i (0 <= i < K/R) reads elements i + r K/R, applies the R-point
// DFT and writes element (i - i mod L) R + (i mod L) + r L.  Thread tau runs
// butterflies tau + g Tn (Tn = K / V threads per sequence, all in one warp).
// IMODE / OMODE: 0 natural positions, 1 Makhoul reordering, 2 swizzled with
// shift SH.  With TWOUT (the first of two passes, L = 1) output r of
// butterfly i is multiplied by exp(-2 pi i r i / K), the twiddle the second
// pass (L = K / R) would apply to its input (i, r) -- the four-step form: the
// factors are read from tw4[r][i] (i contiguous) as each output is stored.
template <int MODE, int K, int SH>
__device__ __forceinline__ int fast_pos(int e) {
  if constexpr (MODE == 1) return makhoul_perm(e, K);
  else if constexpr (MODE == 2) return e ^ ((e >> SH) & ((1 << (SH < 4 ? SH : 4)) - 1));
  else return e;
}

template <typename T, int R, int V, int K, int L, int IMODE, int OMODE, bool TWOUT, int SH, int QP>
__device__ __forceinline__ void fast_pass(cpx<T>* base, bool active, int tau, const cpx<T>* tw4) {
  constexpr int Tn = K / V, G = V / R, KR = K / R, Qp = QP;
  static_assert(Tn <= 32, "a sequence must fit one warp");
  static_assert(!TWOUT || L == 1, "four-step twiddles follow the first pass");
  cpx<T> u[V];
  if (active) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int i = tau + g * Tn;
#pragma unroll
      for (int r = 0; r < R; ++r) u[g * R + r] = base[fast_pos<IMODE, K, SH>(i + r * KR) * Qp];
    }
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int i = tau + g * Tn;
      const int k = i & (L - 1);
      Dft<T, R>::run(&u[g * R]);
      const int j0 = (i - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cpx<T> v = u[g * R + r];
        if constexpr (TWOUT) {
          if (r > 0) v = cmul(v, ld_cpx<T>(tw4, r * KR + i));
        }
        base[fast_pos<OMODE, K, SH>(j0 + r * L) * Qp] = v;
      }
    }
  }
  __syncwarp();
}

// All W * Q sequences of the tile: forward DFT of length K = R0 R1 (R1 = 1:
// one pass), in place.  PIN: the first pass reads in Makhoul order (DCT-II
// input); POUT: the last pass writes in Makhoul order (DCT-III output).
template <typename T, int Q, int V, int K, int R0, int R1, int SH, bool PIN, bool POUT>
__device__ void fast_fft_k(cpx<T>* sm, const FastParams& P) {
  constexpr int Tn = K / V;
  const int W = P.g.W;
  const int nseq = W * Q;
  const int spr = blockDim.x / Tn;
  const int sl = threadIdx.x / Tn, tau = threadIdx.x - sl * Tn;
  const int rounds = (nseq + spr - 1) / spr;
  const cpx<T>* tw2 = reinterpret_cast<const cpx<T>*>(P.tw2);
  asm volatile("" : "+l"(tw2));
  for (int rd = 0; rd < rounds; ++rd) {
    const int seq = rd * spr + sl;
    const bool active = seq < nseq;
    cpx<T>* base = sm;
    if (active) {
      int pen, q;
      if (P.seq_order == 0) {
        pen = seq / Q;
        q = seq - pen * Q;
      } else {
        q = seq / W;
        pen = seq - q * W;
      }
      base = sm + pen * P.pitch + q;
    }
    if constexpr (R1 == 1) {
      fast_pass<T, R0, V, K, 1, PIN ? 1 : 0, POUT ? 1 : 0, false, SH, Q | 1>(base, active, tau, tw2);
    } else {
      fast_pass<T, R0, V, K, 1, PIN ? 1 : 0, 2, true, SH, Q | 1>(base, active, tau, tw2);
      fast_pass<T, R1, V, K, R0, 2, POUT ? 1 : 0, false, SH, Q | 1>(base, active, tau, tw2);
    }
  }
}

// The schedules of fast_schedule: V = 32 for K = 1024 (32 x 32) and 512
// (32 x 16); V = 16 for K = 256 (16 x 16) down to 16 (one pass).  The swizzle
// shift of the exchange buffer (fast_swizzle_shift) is chosen per schedule by
// the bank model of pencil_fast_plan.cpp.
template <typename T, int Q, int V, bool PIN, bool POUT>
__device__ void fast_fft(cpx<T>* sm, const FastParams& P) {
  if constexpr (V == 32) {
    if (P.K == 1024) fast_fft_k<T, Q, 32, 1024, 32, 32, 5, PIN, POUT>(sm, P);
    else fast_fft_k<T, Q, 32, 512, 32, 16, 5, PIN, POUT>(sm, P);
  } else {
    switch (P.K) {
      case 256: fast_fft_k<T, Q, 16, 256, 16, 16, 4, PIN, POUT>(sm, P); break;
      case 128: fast_fft_k<T, Q, 16, 128, 16, 8, 3, PIN, POUT>(sm, P); break;
      case 64: fast_fft_k<T, Q, 16, 64, 16, 4, 2, PIN, POUT>(sm, P); break;
      case 32: fast_fft_k<T, Q, 16, 32, 16, 2, 2, PIN, POUT>(sm, P); break;
      default: fast_fft_k<T, Q, 16, 16, 16, 1, 0, PIN, POUT>(sm, P); break;
    }
  }
}

// ------------------------------------------------------ loads and stores

template <int NORD, int Q2P>
__device__ __forceinline__ int fast_slot(int j) {
  const int e = j / NORD;
  return e * Q2P + (j - e * NORD);
}

// Asynchronous 4-byte global -> shared copy (cp.async, no register staging);
// completed by fast_copy_wait.
__device__ __forceinline__ void fast_copy4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void fast_copy_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Global -> shared: element i of pencil p goes to real slot fast_slot(i)
// (field) or fast_slot(i + 1) (spectral) of the pencil.  Contiguous pencils
// are swept by the whole block; the W pencils of a strided tile are adjacent
// in memory, thread t serving pencil t mod W.  float32 fields are copied
// with cp.async, the whole tile in flight at once; float64 fields (rounded
// to T) go through registers, LB loads in flight per thread, and are checked
// for NaN and Inf (the return value).  Elements of pencils beyond the array
// are not loaded (their results are not stored).
template <typename T, int NORD, bool NC, int LB>
__device__ bool fast_load(T* smr, const FastParams& P, long long tile, bool spectral) {
  bool nf = false;   // a float64 input value that is not finite
  const bool check = P.nonfinite != nullptr;
  const PassGeom& g = P.g;
  constexpr int Q2p = 2 * ((NORD / 2 + 1) | 1);
  const int M = g.M, P2 = 2 * P.pitch;
  const int sh = spectral ? 1 : 0;
  const bool async = !P.in_f64 && sizeof(T) == 4;
  const float* inf = reinterpret_cast<const float*>(P.in);
  const double* ind = reinterpret_cast<const double*>(P.in);
  if (g.inner == 1) {
    for (int p = 0; p < g.W; ++p) {
      const long long base = pencil_base(g, tile, p);
      if (base < 0) continue;
      T* dst = smr + p * P2;
      if (async) {
        for (int i = threadIdx.x; i < M; i += blockDim.x) fast_copy4(dst + fast_slot<NORD, Q2p>(i + sh), inf + base + i);
        continue;
      }
      for (int i0 = threadIdx.x; i0 < M; i0 += LB * blockDim.x) {
        // every load of the batch is issued before any value is converted
        double x[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int i = i0 + u * blockDim.x;
          x[u] = i < M ? ld_field<NC>(ind + base + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int i = i0 + u * blockDim.x;
          if (check) nf |= nonfinite_f64(x[u]);
          T v;
          from_f64(x[u], v);
          if (i < M) dst[fast_slot<NORD, Q2p>(i + sh)] = v;
        }
      }
    }
    if (async) fast_copy_wait();
    return nf;
  }
  const int W = g.W;
  const int p = threadIdx.x & (W - 1);
  const int istep = blockDim.x / W;
  const long long base = pencil_base(g, tile, p);
  const long long stride = g.inner;
  T* dst = smr + p * P2;
  if (base < 0) return nf;
  if (async) {
    for (int i = threadIdx.x / W; i < M; i += istep)
      fast_copy4(dst + fast_slot<NORD, Q2p>(i + sh), inf + base + (long long)i * stride);
    fast_copy_wait();
    return nf;
  }
  for (int i0 = threadIdx.x / W; i0 < M; i0 += LB * istep) {
    double x[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int i = i0 + u * istep;
      x[u] = i < M ? ld_field<NC>(ind + base + (long long)i * stride) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int i = i0 + u * istep;
      if (check) nf |= nonfinite_f64(x[u]);
      T v;
      from_f64(x[u], v);
      if (i < M) dst[fast_slot<NORD, Q2p>(i + sh)] = v;
    }
  }
  return nf;
}

// Shared -> global.  With accumulation (u += result) the old values are
// loaded SB at a time before any of the batch is stored.
template <typename T, int NORD, bool NC>
__device__ void fast_store(const T* smr, const FastParams& P, long long tile, bool spectral) {
  constexpr int SB = 8;
  const PassGeom& g = P.g;
  constexpr int Q2p = 2 * ((NORD / 2 + 1) | 1);
  const int M = g.M, P2 = 2 * P.pitch;
  const int sh = spectral ? 1 : 0;
  const int W = g.W;
  const bool contig = g.inner == 1;
  const int np = contig ? W : 1;
  const int istep = contig ? blockDim.x : blockDim.x / W;
  const int i00 = contig ? threadIdx.x : threadIdx.x / W;
  const long long stride = contig ? 1 : g.inner;
  for (int pp = 0; pp < np; ++pp) {
    const int p = contig ? pp : (threadIdx.x & (W - 1));
    const long long base = pencil_base(g, tile, p);
    if (base < 0) continue;
    const T* src = smr + p * P2;
    if (P.out_f64) {
      double* o = reinterpret_cast<double*>(P.out) + base;
      for (int i0 = i00; i0 < M; i0 += SB * istep) {
        double old[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
          const int i = i0 + u * istep;
          old[u] = 0.0;
          if (P.accum && i < M) old[u] = NC ? o[(long long)i * stride] : __ldcg(o + (long long)i * stride);
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
          const int i = i0 + u * istep;
          if (i < M) {
            const double v = to_f64(src[fast_slot<NORD, Q2p>(i + sh)]);
            o[(long long)i * stride] = P.accum ? old[u] + v : v;   // one float64 add when accumulating
          }
        }
      }
    } else {
      float* o = reinterpret_cast<float*>(P.out) + base;
      for (int i0 = i00; i0 < M; i0 += SB * istep) {
        float old[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
          const int i = i0 + u * istep;
          old[u] = 0.0f;
          if (P.accum && i < M) old[u] = NC ? o[(long long)i * stride] : __ldcg(o + (long long)i * stride);
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
          const int i = i0 + u * istep;
          if (i < M) o[(long long)i * stride] = old[u] + float(src[fast_slot<NORD, Q2p>(i + sh)]);
        }
      }
    }
  }
}

// ------------------------------------------- sequence build / reconstruct

// Chunk e of every pencil: its n fine-grid reals -> the Q packed complex
// values (q = 0: node sum and difference, q >= 1: y[q-1] +- y[n-q-1]; sine
// parts modulated by (-1)^e), in place.  The left node of element e is the
// last real of chunk e-1, read before any chunk is rewritten.
template <typename T, int NORD>
__device__ void fast_build(cpx<T>* sm, const FastParams& P) {
  constexpr int Q = NORD / 2 + 1;
  constexpr int Qp = Q | 1;
  const int K = P.K;
  const int kshift = __ffs(K) - 1;
  const int nchunks = P.g.W * K;
  T xl[kFastChunkTasks];
#pragma unroll
  for (int t = 0; t < kFastChunkTasks; ++t) {
    const int c = threadIdx.x + t * blockDim.x;
    xl[t] = T(0);
    if (c < nchunks) {
      const int p = c >> kshift, e = c & (K - 1);
      if (e > 0) xl[t] = reinterpret_cast<const T*>(sm + p * P.pitch + (e - 1) * Qp)[NORD - 1];
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kFastChunkTasks; ++t) {
    const int c = threadIdx.x + t * blockDim.x;
    if (c < nchunks) {
      const int p = c >> kshift, e = c & (K - 1);
      cpx<T>* ch = sm + p * P.pitch + e * Qp;
      T y[2 * Q];   // the chunk read in (re, im) pairs: 2Q >= n reals
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const cpx<T> v = ch[q];
        y[2 * q] = v.re;
        y[2 * q + 1] = v.im;
      }
      const T xr = (e < K - 1) ? y[NORD - 1] : T(0);
      const T sg = (e & 1) ? T(-1) : T(1);
      cpx<T> out[Q];
      out[0] = {sg * (xr + xl[t]), xr - xl[t]};
#pragma unroll
      for (int q = 1; q < Q; ++q) {
        if (2 * q < NORD) out[q] = {sg * (y[q - 1] + y[NORD - q - 1]), y[q - 1] - y[NORD - q - 1]};
        else out[q] = {sg * y[q - 1], T(0)};
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) ch[q] = out[q];
    }
  }
  __syncthreads();
}

// DCT-III outputs x_e[q] (sine part (-1)^e Re, cosine part Im) -> the n
// fine-grid reals of element e, in place.
template <typename T, int NORD>
__device__ void fast_reconstruct(cpx<T>* sm, const FastParams& P) {
  constexpr int Q = NORD / 2 + 1;
  constexpr int Qp = Q | 1;
  const int K = P.K;
  const int kshift = __ffs(K) - 1;
  const int nchunks = P.g.W * K;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) {
    const int p = c >> kshift, e = c & (K - 1);
    cpx<T>* ch = sm + p * P.pitch + e * Qp;
    cpx<T> x[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) x[q] = ch[q];
    const T sg = (e & 1) ? T(-1) : T(1);
    T y[2 * Q];   // written back in (re, im) pairs; y[n] (n odd) is padding
    y[2 * Q - 1] = T(0);
    y[NORD - 1] = sg * x[0].re + x[0].im;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
      const T ys = sg * x[q].re, yc = x[q].im;
      if (2 * q < NORD) {
        y[q - 1] = ys + yc;
        y[NORD - q - 1] = ys - yc;
      } else {
        y[q - 1] = ys;
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) ch[q] = cpx<T>{y[2 * q], y[2 * q + 1]};
  }
  __syncthreads();
}

// ------------------------------------------------------------ maps

__device__ __forceinline__ float fast_div(float x, float d) { return __fdividef(x, d); }
__device__ __forceinline__ double fast_div(double x, double d) { return divide_by(x, d); }

// The maps of one frequency k (Theorem 2): X (2Q reals: doubled sine and
// cosine sums of the Q sequences, or for k = 0 the plain alternating / plain
// sums) -> coefficients c_l = (1/N_kl) sum_j c_j G_k[j][l] X_j, optionally
// divided by den_base + mu(k, l); then (fused) the inverse map
// out_j = sum_l G_k[j][l] c_l.  nl = n (k >= 1) or n - 1 (bubble modes).
template <typename T, int NORD, int K>
__device__ __forceinline__ void fast_forward_map(const T* X, int k, const T* G, const T* IN, T* c, int nl) {
  constexpr int Q2 = 2 * (NORD / 2 + 1);
#pragma unroll
  for (int l = 0; l < NORD; ++l) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < Q2; ++j) acc = fmaT(__ldg(&G[((size_t)j * NORD + l) * K + k]), X[j], acc);
    c[l] = l < nl ? acc * __ldg(&IN[(size_t)l * K + k]) : T(0);
  }
}
template <typename T, int NORD, int K>
__device__ __forceinline__ void fast_inverse_map(const T* c, int k, const T* G, T* out) {
  constexpr int Q2 = 2 * (NORD / 2 + 1);
#pragma unroll
  for (int j = 0; j < Q2; ++j) {
    T acc = T(0);
#pragma unroll
    for (int l = 0; l < NORD; ++l) acc = fmaT(__ldg(&G[((size_t)j * NORD + l) * K + k]), c[l], acc);
    out[j] = acc;
  }
}

// One thread per (frequency pair, pencil): pairs (k, K-k) for k = 1..K/2-1;
// task 0 handles k = 0 (bubble modes, Theorem 2 first formulas) and the
// self-paired k = K/2.  MODE_FWD: FFT output -> coefficients (spectral
// slots); MODE_INV: coefficients -> pre-twiddled DCT-III input; MODE_FUSED:
// both with the division in between.
template <typename T, int NORD, int MODE, int K>
__device__ void fast_maps(cpx<T>* sm, const FastParams& P, const T* den_base) {
  constexpr int Q = NORD / 2 + 1, Q2 = 2 * Q;
  constexpr int Qp = Q | 1;
  const int W = P.g.W;
  const int half = K >> 1;
  const int ntask = W * half;
  const T* G = reinterpret_cast<const T*>(P.gmap);
  const T* IN = reinterpret_cast<const T*>(P.invn);
  const T* MU = reinterpret_cast<const T*>(P.muk);
  const cpx<T>* rot = reinterpret_cast<const cpx<T>*>(P.rot);
  // opaque to loop-invariant code motion: inside the persistent tile loop
  // the compiler would otherwise keep every table address live across tiles
  asm volatile("" : "+l"(G), "+l"(IN), "+l"(MU), "+l"(rot));
  constexpr bool FWD = MODE != MODE_INV;
  constexpr bool INV = MODE != MODE_FWD;
  for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
    const int tau = task / W;
    const int p = task - tau * W;
    cpx<T>* pen = sm + p * P.pitch;
    const T dbase = INV && FWD ? den_base[p] : T(0);
    // two frequencies per task: (k1, k2) = (tau, K - tau), or (0, K/2)
    const int k1 = tau, k2 = tau ? K - tau : half;
    T X1[Q2], X2[Q2];
    const cpx<T> rk = ld_cpx<T>(rot, tau ? tau : half);
    if (FWD) {
      cpx<T> v1[Q], v2[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        v1[q] = pen[k1 * Qp + q];
        v2[q] = pen[k2 * Qp + q];
      }
      if (tau) {
        // post-twiddle of the DCT-II: A = e^{-i phi_k} V_k, B = e^{+i phi_k} V_{K-k}
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const cpx<T> A = cmul(rk, v1[q]);
          const cpx<T> B = cmul(cpx<T>{rk.re, -rk.im}, v2[q]);
          X1[2 * q] = B.im - A.im;
          X1[2 * q + 1] = A.im + B.im;
          X2[2 * q] = A.re + B.re;
          X2[2 * q + 1] = A.re - B.re;
        }
      } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          X1[2 * q] = v1[q].re;       // S_q(K), C_q(0): the bubble sums
          X1[2 * q + 1] = v1[q].im;
          const cpx<T> A = cmul(rk, v2[q]);
          const cpx<T> B = cmul(cpx<T>{rk.re, -rk.im}, v2[q]);
          X2[2 * q] = B.im - A.im;
          X2[2 * q + 1] = A.im + B.im;
        }
      }
      // c_j = 1/2 on the node slots (the bubble maps are zero there)
      X1[0] *= T(0.5);
      X1[1] *= T(0.5);
      X2[0] *= T(0.5);
      X2[1] *= T(0.5);
    } else {
      // spectral coefficients of the two frequencies (k = 0: slots 1..n-1)
      const T* c1 = reinterpret_cast<const T*>(pen + k1 * Qp);
      const T* c2 = reinterpret_cast<const T*>(pen + k2 * Qp);
#pragma unroll
      for (int l = 0; l < NORD; ++l) {
        X1[l] = tau ? c1[l] : (l + 1 < NORD ? c1[l + 1] : T(0));
        X2[l] = c2[l];
      }
    }
    T c[NORD];
    T o1[Q2], o2[Q2];
    // frequency k1
    if (FWD) {
      fast_forward_map<T, NORD, K>(X1, k1, G, IN, c, tau ? NORD : NORD - 1);
      if (INV) {
#pragma unroll
        for (int l = 0; l < NORD; ++l) {
          const int nl = tau ? NORD : NORD - 1;
          c[l] = l < nl ? fast_div(c[l], dbase + __ldg(&MU[(size_t)l * K + k1])) : T(0);
        }
      }
    } else {
#pragma unroll
      for (int l = 0; l < NORD; ++l) c[l] = X1[l];
    }
    if (INV) {
      fast_inverse_map<T, NORD, K>(c, k1, G, o1);
    } else {
      T* c1 = reinterpret_cast<T*>(pen + k1 * Qp);
#pragma unroll
      for (int l = 0; l < NORD; ++l)
        if (tau) c1[l] = c[l];
        else if (l + 1 < NORD) c1[l + 1] = c[l];
    }
    // frequency k2
    if (FWD) {
      fast_forward_map<T, NORD, K>(X2, k2, G, IN, c, NORD);
      if (INV) {
#pragma unroll
        for (int l = 0; l < NORD; ++l) c[l] = fast_div(c[l], dbase + __ldg(&MU[(size_t)l * K + k2]));
      }
    } else {
#pragma unroll
      for (int l = 0; l < NORD; ++l) c[l] = X2[l];
    }
    if (INV) {
      fast_inverse_map<T, NORD, K>(c, k2, G, o2);
    } else {
      T* c2 = reinterpret_cast<T*>(pen + k2 * Qp);
#pragma unroll
      for (int l = 0; l < NORD; ++l) c2[l] = c[l];
    }
    if (INV) {
      // pre-twiddle of the DCT-III: with (a, b) = (out[2q], out[2q+1]),
      // H_k = e^{-i phi_k} ((a(K-k) - b(K-k)) + i (a(k) + b(k))),
      // H_{K-k} = -i e^{+i phi_k} ((a(k) - b(k)) + i (a(K-k) + b(K-k)));
      // k = 0: H_0 = a(K) + i b(0); k = K/2: H = e^{-i phi} ((a - b) + i (a + b))
      const cpx<T> rc = {-rk.im, -rk.re};   // -i conj(rk)
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const T a1 = o1[2 * q], b1 = o1[2 * q + 1], a2 = o2[2 * q], b2 = o2[2 * q + 1];
        if (tau) {
          pen[k1 * Qp + q] = cmul(rk, cpx<T>{a2 - b2, a1 + b1});
          pen[k2 * Qp + q] = cmul(rc, cpx<T>{a1 - b1, a2 + b2});
        } else {
          pen[k1 * Qp + q] = cpx<T>{a1, b1};
          pen[k2 * Qp + q] = cmul(rk, cpx<T>{a2 - b2, a2 + b2});
        }
      }
    }
  }
  __syncthreads();
}

// The map phase for the K of the tile (compile-time K: every table offset is
// an immediate of the load).
template <typename T, int NORD, int MODE, int V>
__device__ __forceinline__ void fast_maps_k(cpx<T>* sm, const FastParams& P, const T* den_base) {
  if constexpr (V == 32) {
    if (P.K == 1024) fast_maps<T, NORD, MODE, 1024>(sm, P, den_base);
    else fast_maps<T, NORD, MODE, 512>(sm, P, den_base);
  } else {
    switch (P.K) {
      case 256: fast_maps<T, NORD, MODE, 256>(sm, P, den_base); break;
      case 128: fast_maps<T, NORD, MODE, 128>(sm, P, den_base); break;
      case 64: fast_maps<T, NORD, MODE, 64>(sm, P, den_base); break;
      case 32: fast_maps<T, NORD, MODE, 32>(sm, P, den_base); break;
      default: fast_maps<T, NORD, MODE, 16>(sm, P, den_base); break;
    }
  }
}

// --------------------------------------------------------- L2 prefetch

// Asynchronous prefetch of [lo, hi) bytes into L2 (cp.async.bulk.prefetch:
// 16-byte aligned start and size).  The range is shrunk to whole 16-byte
// granules inside [lo, hi) plus the granule holding lo, so that nothing
// outside the array's allocation is touched.
__device__ __forceinline__ void l2_prefetch(const char* lo, const char* hi, const char* arr_end) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(lo) & ~uintptr_t(15);
  uintptr_t b = (reinterpret_cast<uintptr_t>(hi) + 15) & ~uintptr_t(15);
  const uintptr_t e = reinterpret_cast<uintptr_t>(arr_end) & ~uintptr_t(15);
  if (b > e) b = e;
  if (b <= a) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(b - a)) : "memory");
}

// Prefetch the elements of tile `tile` of an array laid out like the pass's
// field (element size es) into L2: one bulk request per contiguous pencil.
__device__ __forceinline__ void fast_prefetch(const FastParams& P, const void* arr, int es, long long tile) {
  const PassGeom& g = P.g;
  if (tile >= g.tiles) return;
  const char* a = reinterpret_cast<const char*>(arr);
  const char* end = a + (size_t)g.outer * g.M * g.inner * es;
  if (g.inner == 1) {
    for (int p = threadIdx.x; p < g.W; p += blockDim.x) {
      const long long base = pencil_base(g, tile, p);
      if (base >= 0) l2_prefetch(a + base * es, a + (base + g.M) * es, end);
    }
    return;
  }
  // strided tiles: one request per element row costs more issue slots than
  // it saves; not prefetched
}

// ------------------------------------------------------------ the pass

template <typename T, int NORD, int MODE, int V, bool NC>
__device__ __forceinline__ void fast_tile(const FastParams& P, long long tile, unsigned char* smem_raw, T* den_base) {
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  T* smr = reinterpret_cast<T*>(smem_raw);
  constexpr int Q = NORD / 2 + 1;
  constexpr int LB = sizeof(T) == 8 ? 8 : 16;
  if (MODE == MODE_FUSED && threadIdx.x < P.g.W) {
    // c + sum over the other axes of a_j mu_j for this pencil (pencil.cuh)
    PassParams Pd;
    Pd.g = P.g;
    Pd.dv = P.dv;
    den_base[threadIdx.x] = pencil_den_base<T, NORD>(Pd, tile, threadIdx.x);
  }
  // the barrier after the load also ORs the non-finite checks of the block
  if (MODE == MODE_INV) {
    const bool nf = fast_load<T, NORD, NC, LB>(smr, P, tile, true);
    if (__syncthreads_or(nf) && threadIdx.x == 0 && P.nonfinite) atomicOr(P.nonfinite, 1);
  } else {
    const bool nf = fast_load<T, NORD, NC, LB>(smr, P, tile, false);
    if (__syncthreads_or(nf) && threadIdx.x == 0 && P.nonfinite) atomicOr(P.nonfinite, 1);
    fast_build<T, NORD>(sm, P);
    fast_fft<T, Q, V, true, false>(sm, P);
    __syncthreads();
  }
  fast_maps_k<T, NORD, MODE, V>(sm, P, den_base);
  if (MODE == MODE_FWD) {
    fast_store<T, NORD, NC>(smr, P, tile, true);
    return;
  }
  fast_fft<T, Q, V, false, true>(sm, P);
  __syncthreads();
  fast_reconstruct<T, NORD>(sm, P);
  fast_store<T, NORD, NC>(smr, P, tile, false);
}

// One tile per CTA.  Before its own tile, a CTA asks L2 for the input of
// the tile `ahead` positions later -- the tile that the CTA taking its place
// on this SM (CTAs start in index order, one per SM at a time) will load --
// and, when the pass accumulates into its output, for its own output rows,
// so that those loads do not wait on HBM latency.  (A persistent loop over
// tiles would do the same but made ptxas spill heavily.)
template <typename T, int NORD, int MODE, int V>
__global__ void __launch_bounds__(fast_threads<V, MODE>(), (fast_min_blocks<V, MODE>())) pencil_fast_kernel(FastParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T den_base[kMaxW];
  const long long tile = blockIdx.x;
  if (P.ahead > 0) fast_prefetch(P, P.in, P.in_f64 ? 8 : 4, tile + P.ahead);
  if (P.accum) fast_prefetch(P, P.out, P.out_f64 ? 8 : 4, tile);
  fast_tile<T, NORD, MODE, V, true>(P, tile, smem_raw, den_base);
}

}  // namespace femfft
