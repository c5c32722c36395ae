// Pencil-pass kernels: the direct FC_n-transform, the inverse F_n-transform
// and the fused forward / spectral-divide / inverse pass along one axis.
//
// Method (Zlotnik & Zlotnik, arXiv:1701.03967, Section 3, Theorem 2 and
// Section 4, algorithm (a)).  For one pencil y in S_K^(n) (node values y_j,
// j = 1..K-1, and element-interior vectors y_{j-1/2} in R^{n-1}) the FC_n
// coefficient of mode (k, l), k >= 1, is (Theorem 2, item 2)
//     y~_kl = [ sum_j y_j sin(pi k j/K)
//             + sum_j y_{j-1/2} . (p sin(pi k (j-1)/K) + flip(p) sin(pi k j/K)) ] / N_kl,
// with p = p_k^(l) and N_kl = ||s_k^(l)||_C^2.  With phi_k = pi k / (2K) and
// the half-sample angles pi k (j - 1/2) / K, the identity used in the proof
// of Theorem 2 gives
//     p sin(pi k (j-1)/K) + flip(p) sin(pi k j/K)
//         = 2 cos(phi_k) p_e sin(pi k (j-1/2)/K) - 2 sin(phi_k) p_o cos(pi k (j-1/2)/K),
// and the node sum is rewritten the same way through the sum and the
// difference of the two nodes of each element:
//     sum_j y_j sin(pi k j/K) = 1/2 cos(phi_k) DST2(y_j + y_{j-1})_k
//                               + 1/2 sin(phi_k) DCT2(y_j - y_{j-1})_k.
// So every coefficient needs only half-sample sine (DST-II) and cosine
// (DCT-II) sums of n+1 real sequences per pencil: the node sum and
// difference, and the even/odd combinations y[m] +- y[n-m] of the interiors.
// The bubble modes (k = 0, Theorem 2, item 2, first formula) are the same
// sums at frequency K (sine: alternating sum) and 0 (cosine: plain sum).
// The inverse F_n-transform (Theorem 2, item 1) is the transpose structure:
// node values by a DST-III plus DCT-III of sigma_k = sum_l w_kl weighted by
// cos(phi_k) / sin(phi_k), interiors by the DST-III of 2cos(phi_k) d_{k,e}
// and the DCT-III of -2 sin(phi_k) d_{k,o} (d_k = sum_l w_kl p_k^(l)), the
// bubble term entering as the k = K sine and k = 0 cosine coefficients.
//
// GPU mapping.  A sine sequence (modulated by (-1)^j) and a cosine sequence
// are packed as the real and imaginary parts of one complex sequence of
// length K; one complex FFT of length K then yields both DCT-II (Makhoul's
// even/odd reordering and a post-twiddle by exp(-i phi_k) combining bins k and
// K-k), and likewise for DCT-III (pre-twiddle, FFT, un-reordering).  A CTA
// holds W whole pencils in shared memory (chunk e of a pencil = element e,
// 2Q reals), builds the Q = floor(n/2)+1 complex sequences in place, runs a
// mixed-radix (2,3,4,8) Stockham FFT with the reorderings folded into the
// first/last pass addressing, and applies the per-frequency n x (n+1) maps
// with one thread per frequency pair (k, K-k).  Everything between the HBM
// load and the HBM store stays in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "femfft_internal.h"

namespace femfft {

template <typename T>
struct cpx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
// multiply by -i
template <typename T>
__device__ __forceinline__ cpx<T> cmi(cpx<T> a) { return {a.im, -a.re}; }

template <typename T>
__device__ __forceinline__ cpx<T> ld_cpx(const void* base, int idx) {
  const T* p = reinterpret_cast<const T*>(base) + 2 * idx;
  return {__ldg(p), __ldg(p + 1)};
}

// float64 <-> float32 by integer bit operations.  GB300 issues about two
// float64 operations per clock per SM, so the conversions at the float64
// inputs and outputs of the float32 passes (and the non-finite test) would
// otherwise take a sizeable share of those passes on the float64 pipe.
// f64_to_f32_bits: round to nearest even; |x| < 2^-126 flushes to a signed
// zero, |x| >= 2^128 (after rounding) gives infinity, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_int(long long xbits) {
  // branch-free (selects only), so that the loads around it stay in flight
  const unsigned long long b = (unsigned long long)xbits;
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned long long m = b & 0x000fffffffffffffull;
  const int fe = e - 1023 + 127;
  unsigned r = ((unsigned)(fe & 0xff) << 23) | (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1fffffffu);
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;   // a carry may reach infinity
  r = fe >= 255 ? 0x7f800000u : r;
  r = fe <= 0 ? 0u : r;
  r = e == 0x7ff ? (0x7f800000u | (m ? 0x00400000u : 0u)) : r;
  return __uint_as_float(sign | r);
}
// the exact float64 value of a float (subnormal floats flush to zero)
__device__ __forceinline__ double f32_to_f64_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  if (e == 0) return __longlong_as_double((long long)s);
  const unsigned long long de = e == 255 ? 0x7ffull : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(s | (de << 52) | m));
}
__device__ __forceinline__ bool f64_nonfinite_int(long long xbits) {
  return ((((unsigned long long)xbits) >> 52) & 0x7ffu) == 0x7ffu;
}
// a float64 field value as T: float by the integer conversion, double as is
__device__ __forceinline__ void from_f64(double x, float& out) { out = f64_to_f32_int(__double_as_longlong(x)); }
__device__ __forceinline__ void from_f64(double x, double& out) { out = x; }
__device__ __forceinline__ bool nonfinite_f64(double x) { return f64_nonfinite_int(__double_as_longlong(x)); }
// T as float64: exact for both
__device__ __forceinline__ double to_f64(float v) { return f32_to_f64_int(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }

// MODE_FWD_DIV: the forward transform with the spectral division, stored in
// spectral order (the fused pass split in two; used by the batched kernel).
enum PassMode { MODE_FWD = 0, MODE_INV = 1, MODE_FUSED = 2, MODE_FWD_DIV = 3 };

constexpr int kMaxV = 12;          // FFT values held per thread
constexpr int kMaxChunkTasks = 8;  // chunks per thread in the sequence build
constexpr int kMaxRadixPasses = 16;
constexpr int kPencilThreads = 512; // threads per CTA of the float pencil passes
constexpr int kPencilThreads64 = 256; // threads per CTA of the double pencil passes
template <typename T>
__host__ __device__ constexpr int pencil_threads() { return sizeof(T) == 8 ? kPencilThreads64 : kPencilThreads; }
// float forward/inverse passes: two resident CTAs per SM (64 registers per
// thread) so that the load/store phase of one overlaps the shared-memory
// phases of the other; the fused pass keeps one CTA with 128 registers
// (measured faster: its map/FFT phases dominate and need the registers)
constexpr int kPencilCtasPerSm = 2;
template <typename T, int MODE>
__host__ __device__ constexpr int pencil_min_blocks() { return (sizeof(T) == 8 || MODE == 2) ? 1 : kPencilCtasPerSm; }
constexpr int kMaxW = 32;           // pencils per CTA (float)
constexpr int kMaxW64 = 8;          // pencils per CTA (double)
constexpr int kSmallW = 4;          // pencil bound of the small-tile kernel variants
template <typename T>
__host__ __device__ constexpr int max_w() { return sizeof(T) == 8 ? kMaxW64 : kMaxW; }

struct PassParams {
  const void* in;
  void* out;
  PassGeom g;
  AxisDev ax;
  DivideDev dv;
  int pitch;         // complex elements per pencil in shared memory
  int V;             // FFT values per thread
  int npass;
  int radix[kMaxRadixPasses];
  // per pass: product of the earlier radices, its mask when a power of two
  // (else -1), and the twiddle stride K / (prod * radix) (set_fft_passes)
  int pprod[kMaxRadixPasses];
  int pmask[kMaxRadixPasses];
  int pstride[kMaxRadixPasses];
  int kshift;        // log2 K when K is a power of two, else -1 (set_fft_passes)
  int in_f64, out_f64, accum;
  int* nonfinite;    // if set: raised (atomicOr 1) when a float64 input value is NaN or Inf
};

// c = q * d + r for the divisors K and K / 2 of the pass, by shifts when K
// is a power of two
__device__ __forceinline__ void divmod_pow(int c, int d, int shift, int& q, int& r) {
  if (shift >= 0) {
    q = c >> shift;
    r = c & (d - 1);
  } else {
    q = c / d;
    r = c - q * d;
  }
}

// ------------------------------------------------------------- radix DFTs
// forward DFT, omega = exp(-2 pi i / R)

template <typename T>
__device__ __forceinline__ void dft2(cpx<T>* u) {
  cpx<T> a = u[0], b = u[1];
  u[0] = cadd(a, b);
  u[1] = csub(a, b);
}
template <typename T>
__device__ __forceinline__ void dft4(cpx<T>* u) {
  cpx<T> t0 = cadd(u[0], u[2]), t1 = csub(u[0], u[2]);
  cpx<T> t2 = cadd(u[1], u[3]), t3 = cmi(csub(u[1], u[3]));
  u[0] = cadd(t0, t2);
  u[2] = csub(t0, t2);
  u[1] = cadd(t1, t3);
  u[3] = csub(t1, t3);
}
template <typename T>
__device__ __forceinline__ void dft3(cpx<T>* u) {
  const T h = T(0.5), s3 = T(0.86602540378443864676372317075294);   // sqrt(3)/2
  cpx<T> t = cadd(u[1], u[2]), d = csub(u[1], u[2]);
  cpx<T> m = {u[0].re - h * t.re, u[0].im - h * t.im};
  cpx<T> r = {s3 * d.im, -s3 * d.re};   // -i sqrt(3)/2 d
  u[0] = cadd(u[0], t);
  u[1] = cadd(m, r);
  u[2] = csub(m, r);
}
template <typename T>
__device__ __forceinline__ void dft8(cpx<T>* u) {
  const T r2 = T(0.70710678118654752440084436210485);
  // stage 1: radix-2 over (j, j+4)
  cpx<T> a0 = cadd(u[0], u[4]), a4 = csub(u[0], u[4]);
  cpx<T> a1 = cadd(u[1], u[5]), a5 = csub(u[1], u[5]);
  cpx<T> a2 = cadd(u[2], u[6]), a6 = csub(u[2], u[6]);
  cpx<T> a3 = cadd(u[3], u[7]), a7 = csub(u[3], u[7]);
  // twiddles w8^j on the odd half: a5 *= w8, a6 *= -i, a7 *= w8^3
  a5 = {r2 * (a5.re + a5.im), r2 * (a5.im - a5.re)};
  a6 = cmi(a6);
  a7 = {r2 * (a7.im - a7.re), -r2 * (a7.re + a7.im)};
  cpx<T> e[4] = {a0, a1, a2, a3}, o[4] = {a4, a5, a6, a7};
  dft4(e);
  dft4(o);
  u[0] = e[0]; u[2] = e[1]; u[4] = e[2]; u[6] = e[3];
  u[1] = o[0]; u[3] = o[1]; u[5] = o[2]; u[7] = o[3];
}

// Complex offset of chunk k within a pencil (chunks are Q complex values
// long; Q is odd for odd n, which keeps the unit-stride passes conflict-free).
// Padding every 16 chunks removed most bank conflicts of the first radix
// pass but cost more in index arithmetic than it saved (measured).
__host__ __device__ __forceinline__ int cofs(int k, int Q) { return k * Q; }
__host__ __device__ __forceinline__ int pencil_pitch_min(int K, int Q) { return cofs(K, Q); }

// Reordering of Makhoul's DCT via FFT: position r of the FFT sequence holds
// element 2r (r < K/2) or element 2(K-1-r)+1 (r >= K/2).
__device__ __forceinline__ int makhoul_perm(int r, int K) {
  return r < (K >> 1) ? 2 * r : 2 * (K - 1 - r) + 1;
}

// One radix-R pass of the Stockham FFT (in place, register staged: every
// thread reads its values, the block synchronises, then every thread writes
// its results).  Butterfly i (0 <= i < K/R) reads elements i + r K/R,
// twiddles them by exp(-2 pi i r (i mod prod) / (prod R)), applies the
// R-point DFT and writes element (i - i mod prod) R + (i mod prod) + r prod.
// Sequence elements are Q complex values apart.
template <typename T, int R, int Q>
__device__ __forceinline__ void fft_pass(cpx<T>* base, bool active, const PassParams& P, const cpx<T>* tw,
                                         int tau, int tps, int prod, int mask, int stride, bool perm_in,
                                         bool perm_out) {
  const int K = P.ax.K;
  const int T_ = K / R;
  const int nb = P.V / R;
  constexpr int GMAX = kMaxV / R;
  cpx<T> u[GMAX * R];
  if (active) {
#pragma unroll
    for (int g = 0; g < GMAX; ++g) {
      if (g < nb) {
        const int i = tau + g * tps;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          int idx = i + r * T_;
          int src = perm_in ? makhoul_perm(idx, K) : idx;
          u[g * R + r] = base[cofs(src, Q)];
        }
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int g = 0; g < GMAX; ++g) {
      if (g < nb) {
        const int i = tau + g * tps;
        const int kk = mask >= 0 ? (i & mask) : i % prod;
        if (prod > 1) {
#pragma unroll
          for (int r = 1; r < R; ++r) u[g * R + r] = cmul(u[g * R + r], tw[r * kk * stride]);
        }
        if (R == 2) dft2(&u[g * R]);
        if (R == 3) dft3(&u[g * R]);
        if (R == 4) dft4(&u[g * R]);
        if (R == 8) dft8(&u[g * R]);
        const int j = (i - kk) * R + kk;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          int dst = j + r * prod;
          if (perm_out) dst = makhoul_perm(dst, K);
          base[cofs(dst, Q)] = u[g * R + r];
        }
      }
    }
  }
  __syncthreads();
}

// Mixed-radix Stockham FFT over nseq complex sequences of length K; sequence
// s = (pencil, q) lives at sm + pencil * pitch + q with stride Q.
// perm_in: the first pass reads element makhoul_perm(idx) (DCT-II input
// reordering); perm_out: the last pass writes element makhoul_perm(idx)
// (DCT-III output reordering).
template <typename T, int Q>
__device__ void fft_all(cpx<T>* sm, const PassParams& P, const cpx<T>* tw, int nseq, bool perm_in, bool perm_out) {
  const int K = P.ax.K;
  const int tps = K / P.V;                  // tasks per sequence
  const int spr = blockDim.x / tps;         // sequences per round (host: >= 1)
  const int seq_local = threadIdx.x / tps;
  const int tau = threadIdx.x - seq_local * tps;
  for (int s0 = 0; s0 < nseq; s0 += spr) {
    const int seq = s0 + seq_local;
    const bool active = (seq_local < spr) && (seq < nseq);
    cpx<T>* base = sm;
    if (active) {
      int pen = seq / Q, q = seq - pen * Q;
      base = sm + pen * P.pitch + q;
    }
    for (int ps = 0; ps < P.npass; ++ps) {
      const int R = P.radix[ps];
      const int prod = P.pprod[ps], mask = P.pmask[ps], stride = P.pstride[ps];
      const bool pin = perm_in && ps == 0, pout = perm_out && ps == P.npass - 1;
      if (R == 8) fft_pass<T, 8, Q>(base, active, P, tw, tau, tps, prod, mask, stride, pin, pout);
      else if (R == 4) fft_pass<T, 4, Q>(base, active, P, tw, tau, tps, prod, mask, stride, pin, pout);
      else if (R == 3) fft_pass<T, 3, Q>(base, active, P, tw, tau, tps, prod, mask, stride, pin, pout);
      else fft_pass<T, 2, Q>(base, active, P, tw, tau, tps, prod, mask, stride, pin, pout);
    }
  }
}

// fine index j (or spectral sigma+1) -> real offset within a pencil
template <int NORD, int Q2>
__device__ __forceinline__ int chunk_slot(int j) {
  int e = j / NORD;
  return 2 * cofs(e, Q2 / 2) + (j - e * NORD);
}

// Global offset of element 0 of pencil p of tile `tile` (or -1 if the pencil
// lies beyond the array); the element stride along the pencil is g.inner.
__device__ __forceinline__ long long pencil_base(const PassGeom& g, long long tile, int p) {
  if (g.inner == 1) {
    long long o = tile * g.W + p;
    return o < g.outer ? o * g.M : -1;
  }
  long long o = tile / g.tiles_inner;
  long long w = (tile - o * g.tiles_inner) * g.W + p;
  return w < g.inner ? o * g.M * g.inner + w : -1;
}

constexpr int kLoadBatch = 8;   // independent global accesses in flight per thread

// j / M for the flat index j of a tile of contiguous pencils (j < 2^24): a
// float product truncated, then corrected by one step each way (the product
// is off by less than one for j below 2^24).
__device__ __forceinline__ int tile_pencil(int j, int M, float invM) {
  int p = (int)((float)j * invM);
  if (p * M > j) --p;
  else if ((p + 1) * M <= j) ++p;
  return p;
}

// Field loads.  NC: through the read-only data cache (the field is not
// written while the kernel runs); otherwise L2-coherent loads (the batched
// kernel reads fields that other CTAs of the same launch wrote).
template <bool NC, typename S>
__device__ __forceinline__ S ld_field(const S* p) {
  if (NC) return __ldg(p);
  return __ldcg(p);
}

// Global -> shared: element i of pencil p goes to chunk slot map(i) (space)
// or map(i+1) (spectral).  Contiguous pencils (inner == 1): each pencil is
// swept by the whole block; strided pencils: the W pencils of an element row
// are adjacent in memory, so thread t serves pencil t mod W (W is a power of
// two dividing the block size).  Loads are issued kLoadBatch at a time.
template <typename T, int NORD, bool NC>
__device__ bool load_tile(T* smr, const PassParams& P, long long tile, bool spectral) {
  bool nf = false;   // a float64 input value that is not finite
  const bool check = P.nonfinite != nullptr;
  constexpr int Q2 = 2 * (NORD / 2 + 1);
  const PassGeom& g = P.g;
  const int M = g.M;
  const int sh = spectral ? 1 : 0;
  const double* ind = reinterpret_cast<const double*>(P.in);
  const float* inf = reinterpret_cast<const float*>(P.in);
  // one batch of kLoadBatch values: all loads issued first, then converted
  // and stored (a conversion between the loads would hold the later ones back)
  auto batch = [&](T* dst, int i0, int istep, long long base, long long stride) {
    if (P.in_f64) {
      double x[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int i = i0 + u * istep;
        x[u] = (i < M && base >= 0) ? ld_field<NC>(ind + base + (long long)i * stride) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int i = i0 + u * istep;
        if (check) nf |= nonfinite_f64(x[u]);
        T v;
        from_f64(x[u], v);
        if (i < M) dst[chunk_slot<NORD, Q2>(i + sh)] = v;
      }
    } else {
      float x[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int i = i0 + u * istep;
        x[u] = (i < M && base >= 0) ? ld_field<NC>(inf + base + (long long)i * stride) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int i = i0 + u * istep;
        if (i < M) dst[chunk_slot<NORD, Q2>(i + sh)] = T(x[u]);
      }
    }
  };
  if (g.inner == 1) {
    // the tile's pencils are one contiguous range of np * M values: swept
    // flat (short pencils would leave most of a per-pencil batch idle)
    const long long first = tile * g.W;
    const int np = (int)min((long long)g.W, g.outer - first);
    const int L = np * M;
    const long long base = first * M;
    const float invM = 1.0f / (float)M;
    for (int j0 = threadIdx.x; j0 < L; j0 += kLoadBatch * blockDim.x) {
      if (P.in_f64) {
        double x[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
          const int j = j0 + u * blockDim.x;
          x[u] = j < L ? ld_field<NC>(ind + base + j) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
          const int j = j0 + u * blockDim.x;
          if (check) nf |= nonfinite_f64(x[u]);
          T v;
          from_f64(x[u], v);
          if (j < L) {
            const int pp = tile_pencil(j, M, invM);
            smr[2 * pp * P.pitch + chunk_slot<NORD, Q2>(j - pp * M + sh)] = v;
          }
        }
      } else {
        float x[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
          const int j = j0 + u * blockDim.x;
          x[u] = j < L ? ld_field<NC>(inf + base + j) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
          const int j = j0 + u * blockDim.x;
          if (j < L) {
            const int pp = tile_pencil(j, M, invM);
            smr[2 * pp * P.pitch + chunk_slot<NORD, Q2>(j - pp * M + sh)] = T(x[u]);
          }
        }
      }
    }
    return nf;
  }
  const int W = g.W;
  const int p = threadIdx.x & (W - 1);
  const int istep = blockDim.x / W;
  const long long base = pencil_base(g, tile, p);
  T* dst = smr + 2 * p * P.pitch;
  for (int i0 = threadIdx.x / W; i0 < M; i0 += kLoadBatch * istep) batch(dst, i0, istep, base, g.inner);
  return nf;
}

template <typename T, bool NC>
__device__ __forceinline__ void store_one(const PassParams& P, long long off, T v) {
  if (P.out_f64) {
    double* o = reinterpret_cast<double*>(P.out) + off;
    *o = P.accum ? (NC ? *o : __ldcg(o)) + to_f64(v) : to_f64(v);
  } else {
    float* o = reinterpret_cast<float*>(P.out) + off;
    *o = P.accum ? (NC ? *o : __ldcg(o)) + float(v) : float(v);
  }
}

template <typename T, int NORD, bool NC>
__device__ void store_tile(const T* smr, const PassParams& P, long long tile, bool spectral) {
  constexpr int Q2 = 2 * (NORD / 2 + 1);
  const PassGeom& g = P.g;
  const int M = g.M;
  const int sh = spectral ? 1 : 0;
  if (g.inner == 1) {   // flat over the tile's contiguous range, as in load_tile
    const long long first = tile * g.W;
    const int np = (int)min((long long)g.W, g.outer - first);
    const int L = np * M;
    const long long base = first * M;
    const float invM = 1.0f / (float)M;
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
      const int pp = tile_pencil(j, M, invM);
      store_one<T, NC>(P, base + j, smr[2 * pp * P.pitch + chunk_slot<NORD, Q2>(j - pp * M + sh)]);
    }
    return;
  }
  const int W = g.W;
  const int p = threadIdx.x & (W - 1);
  const int istep = blockDim.x / W;
  const long long base = pencil_base(g, tile, p);
  if (base < 0) return;
  const long long stride = g.inner;
  const T* src = smr + 2 * p * P.pitch;
  for (int i = threadIdx.x / W; i < M; i += istep)
    store_one<T, NC>(P, base + (long long)i * stride, src[chunk_slot<NORD, Q2>(i + sh)]);
}

// Build the Q packed complex sequences of every pencil in place:
// q = 0: (node sum, node difference); q = m: (y[m] + y[n-m], y[m] - y[n-m]);
// the sine (real) parts modulated by (-1)^e (DST-II via DCT-II).
template <typename T, int NORD>
__device__ void build_sequences(cpx<T>* sm, const PassParams& P) {
  constexpr int Q = NORD / 2 + 1;
  const int K = P.ax.K;
  const int nchunks = P.g.W * K;
  T xl[kMaxChunkTasks];
#pragma unroll
  for (int t = 0; t < kMaxChunkTasks; ++t) {
    int c = threadIdx.x + t * blockDim.x;
    xl[t] = T(0);
    if (c < nchunks) {
      int p, e;
      divmod_pow(c, K, P.kshift, p, e);
      const T* smr = reinterpret_cast<const T*>(sm + p * P.pitch);
      if (e > 0) xl[t] = smr[2 * cofs(e - 1, Q) + (NORD - 1)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kMaxChunkTasks; ++t) {
    int c = threadIdx.x + t * blockDim.x;
    if (c < nchunks) {
      int p, e;
      divmod_pow(c, K, P.kshift, p, e);
      T* smr = reinterpret_cast<T*>(sm + p * P.pitch) + 2 * cofs(e, Q);
      T y[NORD];
      {
        // the chunk starts on a complex boundary: read it in (re, im) pairs
        const cpx<T>* cv = reinterpret_cast<const cpx<T>*>(smr);
#pragma unroll
        for (int s = 0; s + 1 < NORD; s += 2) {
          const cpx<T> c2 = cv[s / 2];
          y[s] = c2.re;
          y[s + 1] = c2.im;
        }
        if (NORD % 2) y[NORD - 1] = smr[NORD - 1];
      }
      T xr = (e < K - 1) ? y[NORD - 1] : T(0);
      T sg = (e & 1) ? T(-1) : T(1);
      cpx<T> out[Q];
      out[0] = {sg * (xr + xl[t]), xr - xl[t]};
#pragma unroll
      for (int q = 1; q < Q; ++q) {
        if (2 * q < NORD) out[q] = {sg * (y[q - 1] + y[NORD - q - 1]), y[q - 1] - y[NORD - q - 1]};
        else out[q] = {sg * y[q - 1], T(0)};
      }
      cpx<T>* dst = reinterpret_cast<cpx<T>*>(smr);
#pragma unroll
      for (int q = 0; q < Q; ++q) dst[q] = out[q];
    }
  }
  __syncthreads();
}

// Reconstruct the fine-grid values of every element from the DCT-III outputs
// x_e[q] (sine part (-1)^e Re, cosine part Im), in place.
template <typename T, int NORD>
__device__ void reconstruct(cpx<T>* sm, const PassParams& P) {
  constexpr int Q = NORD / 2 + 1;
  const int K = P.ax.K;
  const int nchunks = P.g.W * K;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) {
    int p, e;
    divmod_pow(c, K, P.kshift, p, e);
    cpx<T>* ch = sm + p * P.pitch + cofs(e, Q);
    cpx<T> x[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) x[q] = ch[q];
    T sg = (e & 1) ? T(-1) : T(1);
    T y[NORD];
    y[NORD - 1] = sg * x[0].re + x[0].im;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
      T ys = sg * x[q].re, yc = x[q].im;
      if (2 * q < NORD) {
        y[q - 1] = ys + yc;
        y[NORD - q - 1] = ys - yc;
      } else {
        y[q - 1] = ys;
      }
    }
    // written back in (re, im) pairs
#pragma unroll
    for (int s = 0; s + 1 < NORD; s += 2) ch[s / 2] = cpx<T>{y[s], y[s + 1]};
    if (NORD % 2) reinterpret_cast<T*>(ch)[NORD - 1] = y[NORD - 1];
  }
  __syncthreads();
}

template <typename T, int NORD>
__device__ __forceinline__ T pencil_den_base(const PassParams& P, long long tile, int p) {
  // c + sum over the other axes of a_j mu_j[sigma_j] for the pencil p of this
  // CTA (fused pass on axis 0: the pencil index is the flat index of the
  // later axes), summed in float64.
  const PassGeom& g = P.g;
  long long w = 0;    // inner == 1: the later axes (if any) all have size 1
  if (g.inner > 1) {
    long long o = tile / g.tiles_inner;
    w = (tile - o * g.tiles_inner) * g.W + p;
    if (w >= g.inner) w = 0;
  }
  double base = P.dv.c;
  if (P.dv.nother == 1) {
    base += double(reinterpret_cast<const T*>(P.dv.mu_o[0])[w]);
  } else if (P.dv.nother == 2) {
    long long i1 = w / P.dv.Mo[1], i2 = w - i1 * P.dv.Mo[1];
    base += double(reinterpret_cast<const T*>(P.dv.mu_o[0])[i1]);
    base += double(reinterpret_cast<const T*>(P.dv.mu_o[1])[i2]);
  }
  return T(base);
}

// Post-twiddle of the forward DCT-II (in place).  For the frequency pair
// (k, K-k) and sequence q, with A = exp(-i phi_k) V_k and
// B = exp(+i phi_k) V_{K-k}:  chunk k <- (2 S_q(k), 2 C_q(k)) =
// (Im B - Im A, Im A + Im B), chunk K-k <- (2 S_q(K-k), 2 C_q(K-k)) =
// (Re A + Re B, Re A - Re B).  Chunk 0 already holds (S_q(K), C_q(0)) =
// (Re V_0, Im V_0).
template <typename T, int NORD>
__device__ void post_twiddle(cpx<T>* sm, const PassParams& P, const cpx<T>* rot) {
  constexpr int Q = NORD / 2 + 1;
  const int K = P.ax.K;
  const int npairs = K / 2;
  const int ntask = P.g.W * npairs * Q;
  for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
    const int r = task / Q;
    const int q = task - r * Q;
    int p, km1;
    divmod_pow(r, npairs, P.kshift - 1, p, km1);
    const int k = 1 + km1;
    cpx<T>* pen = sm + p * P.pitch;
    const int kk = K - k;
    const cpx<T> rk = rot[k];
    const cpx<T> A = cmul(rk, pen[cofs(k, Q) + q]);
    const cpx<T> B = cmul(cpx<T>{rk.re, -rk.im}, pen[cofs(kk, Q) + q]);
    pen[cofs(k, Q) + q] = {B.im - A.im, A.im + B.im};
    if (kk != k) pen[cofs(kk, Q) + q] = {A.re + B.re, A.re - B.re};
  }
  __syncthreads();
}

// Per-frequency forward maps (Theorem 2, item 2): coefficient (k, l) =
// F_k[l] . (chunk k slots), for every pencil of the CTA; optionally divided
// by the spectral denominator.  One thread per (k, l) loads the map row once
// (coalesced) and applies it to all W pencils.  Rounds cover whole
// frequencies so that every chunk is read completely before it is rewritten.
// Division by a spectral denominator.  float64: Newton-Raphson reciprocal
// (two steps from the float32 reciprocal, relative error ~2^-96 before the
// final rounding), far cheaper than a float64 division on this GPU.
__device__ __forceinline__ float divide_by(float x, float d) { return x / d; }
__device__ __forceinline__ double divide_by(double x, double d) {
  double r = double(__frcp_rn(float(d)));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  return x * r;
}

// Per-frequency forward maps (Theorem 2, item 2): coefficient (k, l) =
// F_k[l] . (chunk k slots), for every pencil of the CTA; optionally divided
// by the spectral denominator.  One thread per (k, l) loads the map row once
// (coalesced) and applies it to all W pencils; the next round's rows are
// prefetched while the current round computes.  Rounds cover whole
// frequencies so that every chunk is read completely before it is rewritten.
template <typename T, int NORD, bool DIVIDE, int WM>
__device__ void forward_map(cpx<T>* sm, const PassParams& P, const T* base) {
  constexpr int Q2 = 2 * (NORD / 2 + 1);
  const int K = P.ax.K;
  const int W = P.g.W;
  const T* F = reinterpret_cast<const T*>(P.ax.fwd);
  const T* mu = reinterpret_cast<const T*>(P.ax.mu);
  const int kpr = blockDim.x / NORD;
  const int kl = threadIdx.x / NORD, l = threadIdx.x - kl * NORD;
  T f[Q2], fn[Q2];
  T m = T(0), mn = T(0);
  auto fetch = [&](int k, T* dst, T& md) {
    if (kl < kpr && k < K) {
#pragma unroll
      for (int j = 0; j < Q2; ++j) dst[j] = __ldg(&F[((size_t)k * NORD + l) * Q2 + j]);
      if (DIVIDE && !(k == 0 && l == NORD - 1)) md = __ldg(&mu[(k == 0) ? l : NORD * k - 1 + l]);
    }
  };
  fetch(kl, f, m);
  for (int k0 = 0; k0 < K; k0 += kpr) {
    const int k = k0 + kl;
    const bool act = kl < kpr && k < K && !(k == 0 && l == NORD - 1);
    fetch(k + kpr, fn, mn);
    T out[WM];
    if (act) {
#pragma unroll
      for (int p = 0; p < WM; ++p) {
        if (p < W) {
          const T* ch = reinterpret_cast<const T*>(sm + p * P.pitch) + 2 * cofs(k, Q2 / 2);
          T acc = T(0);
#pragma unroll
          for (int j = 0; j < Q2; ++j) acc += f[j] * ch[j];
          if (DIVIDE) acc = divide_by(acc, base[p] + m);
          out[p] = acc;
        }
      }
    }
    __syncthreads();
    if (act) {
      const int slot = (k == 0) ? l + 1 : l;
#pragma unroll
      for (int p = 0; p < WM; ++p)
        if (p < W) reinterpret_cast<T*>(sm + p * P.pitch)[2 * cofs(k, Q2 / 2) + slot] = out[p];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < Q2; ++j) f[j] = fn[j];
    m = mn;
  }
}

// Per-frequency inverse maps (Theorem 2, item 1): chunk k slot j <- I_k[j] .
// w_k, where w_k are the n spectral values of frequency k (slots 0..n-1, or
// 1..n-1 for the bubble modes of k = 0).  Slot 2q receives half the sine
// coefficient a_q, slot 2q+1 half the cosine coefficient b_q of sequence q.
template <typename T, int NORD, int WM>
__device__ void inverse_map(cpx<T>* sm, const PassParams& P) {
  constexpr int Q2 = 2 * (NORD / 2 + 1);
  const int K = P.ax.K;
  const int W = P.g.W;
  const T* I = reinterpret_cast<const T*>(P.ax.inv);
  const int kpr = blockDim.x / Q2;
  const int kl = threadIdx.x / Q2, j = threadIdx.x - kl * Q2;
  T f[NORD], fn[NORD];
  auto fetch = [&](int k, T* dst) {
    if (kl < kpr && k < K) {
#pragma unroll
      for (int l = 0; l < NORD; ++l) dst[l] = __ldg(&I[((size_t)k * Q2 + j) * NORD + l]);
    }
  };
  fetch(kl, f);
  for (int k0 = 0; k0 < K; k0 += kpr) {
    const int k = k0 + kl;
    const bool act = kl < kpr && k < K;
    fetch(k + kpr, fn);
    T out[WM];
    if (act) {
      const int off = (k == 0) ? 1 : 0;
      const int nl = (k == 0) ? NORD - 1 : NORD;
#pragma unroll
      for (int p = 0; p < WM; ++p) {
        if (p < W) {
          const T* ch = reinterpret_cast<const T*>(sm + p * P.pitch) + 2 * cofs(k, Q2 / 2) + off;
          T acc = T(0);
#pragma unroll
          for (int l = 0; l < NORD; ++l)
            if (l < nl) acc += f[l] * ch[l];
          out[p] = acc;
        }
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int p = 0; p < WM; ++p)
        if (p < W) reinterpret_cast<T*>(sm + p * P.pitch)[2 * cofs(k, Q2 / 2) + j] = out[p];
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < NORD; ++l) f[l] = fn[l];
  }
}

// Pre-twiddle of the inverse DCT-III (in place).  With a_q, b_q the halved
// sine/cosine coefficients in slots (2q, 2q+1) of chunks k and K-k:
//   H_k     = exp(-i phi_k)     [(a(K-k) - b(K-k)) + i (a(k) + b(k))],
//   H_{K-k} = exp(-i phi_{K-k}) [(a(k) - b(k)) + i (a(K-k) + b(K-k))],
// exp(-i phi_{K-k}) = -i exp(+i phi_k).  Chunk 0 already holds
// H_0 = a_q(K) + i b_q(0).
template <typename T, int NORD>
__device__ void pre_twiddle(cpx<T>* sm, const PassParams& P, const cpx<T>* rot) {
  constexpr int Q = NORD / 2 + 1;
  const int K = P.ax.K;
  const int npairs = K / 2;
  const int ntask = P.g.W * npairs * Q;
  for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
    const int r = task / Q;
    const int q = task - r * Q;
    int p, km1;
    divmod_pow(r, npairs, P.kshift - 1, p, km1);
    const int k = 1 + km1;
    cpx<T>* pen = sm + p * P.pitch;
    const int kk = K - k;
    const cpx<T> rk = rot[k];
    const cpx<T> vk = pen[cofs(k, Q) + q];      // (a(k), b(k))
    const cpx<T> vkk = pen[cofs(kk, Q) + q];    // (a(K-k), b(K-k))
    pen[cofs(k, Q) + q] = cmul(rk, cpx<T>{vkk.re - vkk.im, vk.re + vk.im});
    if (kk != k) pen[cofs(kk, Q) + q] = cmul(cmi(cpx<T>{rk.re, -rk.im}), cpx<T>{vk.re - vk.im, vkk.re + vkk.im});
  }
  __syncthreads();
}

// One tile of a pencil pass: W pencils loaded, transformed and stored.
// smem_raw holds the pencils (W * pitch complex values) followed by the FFT
// twiddles and DCT rotations (K complex values each), which are staged from
// global memory unless stage_tables is false (the caller guarantees they are
// still in place from the previous tile of the same pass).  base[] receives
// the per-pencil denominator offsets of the fused pass.
template <typename T, int NORD, int MODE, int WM, bool NC>
__device__ __forceinline__ void pencil_tile(const PassParams& P, long long tile, unsigned char* smem_raw, T* base,
                                            bool stage_tables) {
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  T* smr = reinterpret_cast<T*>(smem_raw);
  constexpr int Q = NORD / 2 + 1;
  const int K = P.ax.K;
  cpx<T>* tw = sm + P.g.W * P.pitch;
  cpx<T>* rot = tw + K;
  if (stage_tables) {
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      tw[i] = ld_cpx<T>(P.ax.tw, i);
      rot[i] = ld_cpx<T>(P.ax.rot, i);
    }
  }
  constexpr bool DIVIDE = MODE == MODE_FUSED || MODE == MODE_FWD_DIV;
  if (DIVIDE && threadIdx.x < P.g.W) base[threadIdx.x] = pencil_den_base<T, NORD>(P, tile, threadIdx.x);
  if (MODE == MODE_INV) {
    const bool nf = load_tile<T, NORD, NC>(smr, P, tile, true);
    if (__syncthreads_or(nf) && threadIdx.x == 0 && P.nonfinite) atomicOr(P.nonfinite, 1);
  } else {
    const bool nf = load_tile<T, NORD, NC>(smr, P, tile, false);
    if (__syncthreads_or(nf) && threadIdx.x == 0 && P.nonfinite) atomicOr(P.nonfinite, 1);
    build_sequences<T, NORD>(sm, P);
    fft_all<T, Q>(sm, P, tw, P.g.W * Q, true, false);
    post_twiddle<T, NORD>(sm, P, rot);
    forward_map<T, NORD, DIVIDE, WM>(sm, P, base);
    if (MODE == MODE_FWD || MODE == MODE_FWD_DIV) {
      store_tile<T, NORD, NC>(smr, P, tile, true);
      return;
    }
  }
  inverse_map<T, NORD, WM>(sm, P);
  pre_twiddle<T, NORD>(sm, P, rot);
  fft_all<T, Q>(sm, P, tw, P.g.W * Q, false, true);
  reconstruct<T, NORD>(sm, P);
  store_tile<T, NORD, NC>(smr, P, tile, false);
}

template <typename T, int NORD, int MODE, int WM>
__global__ void __launch_bounds__(pencil_threads<T>(), (pencil_min_blocks<T, MODE>())) pencil_pass_kernel(PassParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T base[WM];
  pencil_tile<T, NORD, MODE, WM, true>(P, blockIdx.x, smem_raw, base, true);
}

}  // namespace femfft
