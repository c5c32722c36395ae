// Pencil passes for long pencils (K too large for one CTA's shared memory,
// up to 2^20 elements): the same transforms as pencil.cuh (Section 3,
// Theorem 2; Section 4, algorithm (a)) staged through a global workspace of
// the Q packed complex sequences of every pencil.
//
//   build:   element e of every pencil -> its Q complex sequence values
//            (node sum/difference, interior even/odd combinations, sine parts
//            times (-1)^e), stored at the Makhoul position of e (DCT-II input
//            order) of sequence q.
//   FFT:     four-step, K = K1 K2, sequences viewed as [K1][K2] row-major.
//            Forward-order input (natural j = j1 K2 + j2): DFT over j1 (the
//            columns), twiddle by exp(-2 pi i j2 k1 / K), DFT over j2 (the
//            rows): X[k1 + K1 k2] lands at [k1][k2] (transposed order).
//            Transposed input (H[a + K1 b] at [a][b]): DFT over b (rows),
//            twiddle exp(-2 pi i a m2 / K), DFT over a (columns): X[m] lands
//            at position m (natural order).  Every stage is a batched
//            shared-memory Stockham FFT of length K1 or K2.
//   maps:    one thread per (pencil, frequency pair (k, K-k)): the DCT
//            post-twiddle, the per-frequency maps of Theorem 2 (the plan's
//            forward and inverse map tables), the division and the DCT-III
//            pre-twiddle, read from and written back to the transposed
//            positions of k and K-k.
//   reconstruct: the DCT-III outputs at the Makhoul positions of element e
//            -> the n fine-grid values of e.
//
// Workspace layouts.  Contiguous pencils (the last axis): S[pencil][q][x],
// a CTA of the FFT stages takes C whole rows or columns of one sequence.
// Strided pencils (an earlier axis, pencil stride `inner`): S[q][x][pencil]
// with the pencils of a group padded to a multiple of 16 (pencil fastest),
// so that the build, map and reconstruct kernels read and write the field
// and the workspace with consecutive threads on consecutive pencils, and an
// FFT CTA takes the same row or column of C adjacent pencils.
// Host code (run_long_pass) at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "plan.h"

namespace femfft {
namespace {

constexpr int kLongThreads = 256;
constexpr int kLongMaxPass = 24;

struct LongFft {
  int L, npass;                 // sequence length of this stage and its radix schedule
  int radix[kLongMaxPass];
  int C;                        // sequences per CTA
  int pitch;                    // complex values per sequence in shared memory
  int cols;                     // 1: DFTs over j1 (stride K2); 0: over j2 (contiguous)
  int twiddle;                  // multiply element (row a, column b) by exp(-2 pi i a b / K) after the DFT
  long long nblocks_per_seq;    // contiguous layout: CTAs per packed sequence (K / L / C)
  // pencil-fastest layout: CTA = (q, line, block of C pencils), lines = the
  // rows or columns of [K1][K2] that the stage does not run along
  int pf, lines, Q;
  long long npad, pblocks;
};

struct LongParams {
  const void* in;
  void* out;
  int in_f64, out_f64, accum;
  void* S;                      // workspace (layout above)
  long long pencils;            // pencils of this group
  long long first;              // index of the group's first pencil (pencil = o * inner + w)
  long long inner;              // element stride of the pencils (1: contiguous)
  int pf;                       // pencil-fastest workspace layout (strided pencils)
  long long npad;               // pf: pencils per workspace row (a multiple of 16)
  int K, K1, K2, M, n;
  const void* tw;               // T2 [K]  exp(-2 pi i j / K)
  const void* rot;              // T2 [K]  exp(-i pi k / (2K))
  const void* fwd;              // T [K][n][2Q]
  const void* inv;              // T [K][2Q][n]
  const void* mu;               // T [M]
  // divisor of the fused pass: c + sum over the later axes of their a s lambda
  // at the pencil's position w (as in the shared-memory passes)
  double c;
  int nother;
  long long Mo[2];
  const void* mu_o[2];
  int* nonfinite;
};

__device__ __forceinline__ int makhoul_inv(int e, int K) { return (e & 1) ? K - 1 - (e >> 1) : (e >> 1); }
__device__ __forceinline__ long long tpos(int k, int K1, int K2) { return (long long)(k % K1) * K2 + k / K1; }

// outer index o and inner position w of the group's pencil pen
__device__ __forceinline__ void pencil_ow(const LongParams& P, long long pen, long long& o, long long& w) {
  const long long gp = P.first + pen;
  if (P.inner == 1) {
    o = gp;
    w = 0;
  } else {
    o = gp / P.inner;
    w = gp - o * P.inner;
  }
}
// field index of position m of the pencil (o, w)
__device__ __forceinline__ long long field_at(const LongParams& P, long long o, long long w, long long m) {
  return (o * P.M + m) * P.inner + w;
}
// workspace index of element x of sequence q of the group's pencil pen
__device__ __forceinline__ long long ws_at(const LongParams& P, int Q, long long pen, int q, long long x) {
  return P.pf ? ((long long)q * P.K + x) * P.npad + pen : (pen * Q + q) * (long long)P.K + x;
}
// (pencil, index) of thread-loop item t over pencils x count items: pencil
// fastest in the pencil-fastest layout, else pencil-major
__device__ __forceinline__ void split_item(const LongParams& P, long long t, long long count, long long& pen,
                                           int& i) {
  if (P.pf) {
    const long long q = t / P.pencils;
    i = (int)q;
    pen = t - q * P.pencils;
  } else {
    pen = t / count;
    i = (int)(t - pen * count);
  }
}
// c + the later axes' eigenvalue terms at the pencil's inner position w
template <typename T>
__device__ __forceinline__ T divisor_base(const LongParams& P, long long w) {
  double b = P.c;
  if (P.nother == 1) {
    b += double(reinterpret_cast<const T*>(P.mu_o[0])[w]);
  } else if (P.nother == 2) {
    const long long i1 = w / P.Mo[1], i2 = w - i1 * P.Mo[1];
    b += double(reinterpret_cast<const T*>(P.mu_o[0])[i1]);
    b += double(reinterpret_cast<const T*>(P.mu_o[1])[i2]);
  }
  return T(b);
}

template <typename T>
__device__ __forceinline__ T load_in(const LongParams& P, long long idx, bool& nf) {
  if (P.in_f64) {
    const double x = reinterpret_cast<const double*>(P.in)[idx];
    if (P.nonfinite) nf |= nonfinite_f64(x);
    T v;
    from_f64(x, v);
    return v;
  }
  return T(reinterpret_cast<const float*>(P.in)[idx]);
}

template <typename T>
__device__ __forceinline__ void store_out(const LongParams& P, long long idx, T v) {
  if (P.out_f64) {
    double* o = reinterpret_cast<double*>(P.out) + idx;
    *o = P.accum ? *o + to_f64(v) : to_f64(v);
  } else {
    float* o = reinterpret_cast<float*>(P.out) + idx;
    *o = P.accum ? *o + float(v) : float(v);
  }
}

// ------------------------------------------------------------------ build

template <typename T, int NORD>
__global__ void __launch_bounds__(kLongThreads) long_build_kernel(LongParams P) {
  constexpr int Q = NORD / 2 + 1;
  const long long total = P.pencils * P.K;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(P.S);
  bool nf = false;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long pen, o, w;
    int e;
    split_item(P, t, P.K, pen, e);
    pencil_ow(P, pen, o, w);
    const long long m0 = (long long)NORD * e;   // first value of element e
    T y[NORD];
#pragma unroll
    for (int s = 0; s < NORD; ++s) {
      const bool last_vertex = (s == NORD - 1) && (e == P.K - 1);   // the right boundary node: not stored
      y[s] = last_vertex ? T(0) : load_in<T>(P, field_at(P, o, w, m0 + s), nf);
    }
    const T xl = e > 0 ? load_in<T>(P, field_at(P, o, w, m0 - 1), nf) : T(0);
    const T xr = y[NORD - 1];
    const T sg = (e & 1) ? T(-1) : T(1);
    const int r = makhoul_inv(e, P.K);
    S[ws_at(P, Q, pen, 0, r)] = cpx<T>{sg * (xr + xl), xr - xl};
#pragma unroll
    for (int q = 1; q < Q; ++q) {
      if (2 * q < NORD) S[ws_at(P, Q, pen, q, r)] = cpx<T>{sg * (y[q - 1] + y[NORD - q - 1]), y[q - 1] - y[NORD - q - 1]};
      else S[ws_at(P, Q, pen, q, r)] = cpx<T>{sg * y[q - 1], T(0)};
    }
  }
  if (__syncthreads_or(nf) && threadIdx.x == 0 && P.nonfinite) atomicOr(P.nonfinite, 1);
}

// -------------------------------------------------------------- FFT stage

// One stage of the four-step FFT: C sequences of length L per CTA, a
// ping-pong Stockham FFT in shared memory (pass s: butterfly i reads
// elements i + r L/R, twiddles them by exp(-2 pi i r (i mod prod) / (prod R)),
// writes element (i - i mod prod) R + i mod prod + r prod), then the
// four-step twiddle.  Column stages (F.cols) run over j1 of [K1][K2]
// (element stride K2), row stages over j2 (contiguous).
template <typename T>
__global__ void __launch_bounds__(kLongThreads) long_fft_kernel(LongParams P, LongFft F) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* B = A + (size_t)F.C * F.pitch;
  const cpx<T>* tw = reinterpret_cast<const cpx<T>*>(P.tw);
  cpx<T>* S = reinterpret_cast<cpx<T>*>(P.S);
  const int K = P.K, L = F.L, C = F.C;
  // element x of local sequence c sits at S[off0 + x xs + c cs]; `other` is
  // the coordinate of [K1][K2] the stage does not run along (row or column)
  long long off0, xs, cs;
  int other0, other_c;   // other = other0 + other_c * c
  if (!F.pf) {
    const long long seq = blockIdx.x / F.nblocks_per_seq;
    const long long blk = blockIdx.x - seq * F.nblocks_per_seq;
    const int c0 = (int)(blk * C);
    off0 = seq * K + (F.cols ? c0 : (long long)c0 * P.K2);
    xs = F.cols ? P.K2 : 1;
    cs = F.cols ? 1 : P.K2;
    other0 = c0;
    other_c = 1;
  } else {
    const long long pb = blockIdx.x % F.pblocks;
    const long long rest = blockIdx.x / F.pblocks;
    const int line = (int)(rest % F.lines);
    const int q = (int)(rest / F.lines);
    const long long x0 = F.cols ? line : (long long)line * P.K2;
    off0 = ((long long)q * K + x0) * F.npad + pb * C;
    xs = (F.cols ? (long long)P.K2 : 1LL) * F.npad;
    cs = 1;
    other0 = line;
    other_c = 0;
  }
  auto goff = [&](int c, int x) -> long long { return off0 + (long long)x * xs + (long long)c * cs; };
  cpx<T>* base = S;
  const bool lanes_c = F.cols || F.pf;   // lanes over c where c is the contiguous index
  for (int t = threadIdx.x; t < C * L; t += blockDim.x) {
    int c, x;
    if (lanes_c) {   // lanes over the C adjacent columns or pencils: coalesced rows
      x = t / C;
      c = t - x * C;
    } else {
      c = t / L;
      x = t - c * L;
    }
    A[c * F.pitch + x] = base[goff(c, x)];
  }
  __syncthreads();
  int prod = 1;
  for (int ps = 0; ps < F.npass; ++ps) {
    const int R = F.radix[ps];
    const int LR = L / R;
    for (int t = threadIdx.x; t < C * LR; t += blockDim.x) {
      const int c = t / LR, i = t - c * LR;
      const int k = i % prod;
      cpx<T> u[8];
      const cpx<T>* src = A + c * F.pitch;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < R) u[r] = src[i + r * LR];
      if (prod > 1) {
        // exp(-2 pi i r k / (prod R)) = tw[r k (K / (prod R))]
        const long long step = (long long)(K / (prod * R)) * k;
#pragma unroll
        for (int r = 1; r < 8; ++r)
          if (r < R) u[r] = cmul(u[r], ld_cpx<T>(tw, (int)((step * r) % K)));
      }
      if (R == 2) dft2(u);
      else if (R == 3) dft3(u);
      else if (R == 4) dft4(u);
      else dft8(u);
      cpx<T>* dst = B + c * F.pitch;
      const int j = (i - k) * R + k;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < R) dst[j + r * prod] = u[r];
    }
    __syncthreads();
    cpx<T>* tmp = A;
    A = B;
    B = tmp;
    prod *= R;
  }
  for (int t = threadIdx.x; t < C * L; t += blockDim.x) {
    int c, x;
    if (lanes_c) {
      x = t / C;
      c = t - x * C;
    } else {
      c = t / L;
      x = t - c * L;
    }
    cpx<T> v = A[c * F.pitch + x];
    if (F.twiddle) {
      // element at (row a, column b) of [K1][K2]: exp(-2 pi i a b / K)
      const long long oth = other0 + (long long)other_c * c;
      const long long a = F.cols ? x : oth, b = F.cols ? oth : x;
      v = cmul(v, ld_cpx<T>(tw, (int)((a * b) % K)));
    }
    base[goff(c, x)] = v;
  }
}

// ------------------------------------------------------------------- maps

// One thread per (pencil, frequency pair): (k, K-k) for k = 1..K/2-1, task
// 0 takes k = 0 (the bubble modes) and the self-paired K/2.  The FFT outputs
// are at the transposed positions of k; FWD writes the FC_n coefficients to
// the output field (spectral layout), INV reads them from the input field,
// FUSED divides by c + mu; INV and FUSED write the pre-twiddled DCT-III
// inputs back to the same positions (transposed order, the input of the
// second FFT).  The maps are the plan's per-frequency tables of Theorem 2.
template <typename T, int NORD, int MODE>
__global__ void __launch_bounds__(kLongThreads) long_map_kernel(LongParams P) {
  constexpr int Q = NORD / 2 + 1, Q2 = 2 * Q;
  constexpr bool FWD = MODE != MODE_INV, INV = MODE != MODE_FWD;
  const int K = P.K, half = K / 2;
  const long long total = P.pencils * half;
  cpx<T>* S = reinterpret_cast<cpx<T>*>(P.S);
  const T* F = reinterpret_cast<const T*>(P.fwd);
  const T* I = reinterpret_cast<const T*>(P.inv);
  const T* mu = reinterpret_cast<const T*>(P.mu);
  const cpx<T>* rot = reinterpret_cast<const cpx<T>*>(P.rot);
  bool nf = false;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long pen, o, w;
    int tau;
    split_item(P, t, half, pen, tau);
    pencil_ow(P, pen, o, w);
    const int k1 = tau, k2 = tau ? K - tau : half;
    const long long p1 = tpos(k1, P.K1, P.K2), p2 = tpos(k2, P.K1, P.K2);
    const cpx<T> rk = ld_cpx<T>(rot, tau ? tau : half);
    T w1[NORD], w2[NORD];                      // the spectral values of k1 and k2
    if (FWD) {
      T X1[Q2], X2[Q2];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const cpx<T> v1 = S[ws_at(P, Q, pen, q, p1)], v2 = S[ws_at(P, Q, pen, q, p2)];
        const cpx<T> A2 = cmul(rk, v2), B2 = cmul(cpx<T>{rk.re, -rk.im}, v2);
        if (tau) {
          const cpx<T> A = cmul(rk, v1);
          X1[2 * q] = B2.im - A.im;
          X1[2 * q + 1] = A.im + B2.im;
          X2[2 * q] = A.re + B2.re;
          X2[2 * q + 1] = A.re - B2.re;
        } else {
          X1[2 * q] = v1.re;
          X1[2 * q + 1] = v1.im;
          X2[2 * q] = B2.im - A2.im;
          X2[2 * q + 1] = A2.im + B2.im;
        }
      }
      const T* F1 = F + (size_t)k1 * NORD * Q2;
      const T* F2 = F + (size_t)k2 * NORD * Q2;
#pragma unroll
      for (int l = 0; l < NORD; ++l) {
        T a1 = T(0), a2 = T(0);
#pragma unroll
        for (int j = 0; j < Q2; ++j) {
          a1 += __ldg(&F1[l * Q2 + j]) * X1[j];
          a2 += __ldg(&F2[l * Q2 + j]) * X2[j];
        }
        w1[l] = a1;
        w2[l] = a2;
      }
      if (tau == 0) {   // bubble coefficients l = 0..n-2
#pragma unroll
        for (int l = NORD - 1; l > 0; --l) w1[l] = w1[l - 1];
        w1[0] = T(0);
      }
      if (MODE == MODE_FWD) {
#pragma unroll
        for (int l = 0; l < NORD; ++l) {
          const int s1 = tau ? NORD * k1 - 1 + l : l - 1;   // spectral index of (k1, l)
          if (s1 >= 0) store_out<T>(P, field_at(P, o, w, s1), w1[l]);
          store_out<T>(P, field_at(P, o, w, (long long)NORD * k2 - 1 + l), w2[l]);
        }
        continue;
      }
      const T b0 = divisor_base<T>(P, w);
#pragma unroll
      for (int l = 0; l < NORD; ++l) {
        const int s1 = tau ? NORD * k1 - 1 + l : l - 1;
        w1[l] = s1 >= 0 ? w1[l] / (b0 + mu[s1]) : T(0);
        w2[l] = w2[l] / (b0 + mu[NORD * k2 - 1 + l]);
      }
    } else {
#pragma unroll
      for (int l = 0; l < NORD; ++l) {
        const int s1 = tau ? NORD * k1 - 1 + l : l - 1;
        w1[l] = s1 >= 0 ? load_in<T>(P, field_at(P, o, w, s1), nf) : T(0);
        w2[l] = load_in<T>(P, field_at(P, o, w, (long long)NORD * k2 - 1 + l), nf);
      }
    }
    if (INV) {
      // inverse maps: out_j = sum_l I_k[j][l] w_l (k = 0: w at slots 1..n-1)
      T o1[Q2], o2[Q2];
      const T* I1 = I + (size_t)k1 * Q2 * NORD;
      const T* I2 = I + (size_t)k2 * Q2 * NORD;
#pragma unroll
      for (int j = 0; j < Q2; ++j) {
        T a1 = T(0), a2 = T(0);
#pragma unroll
        for (int l = 0; l < NORD; ++l) {
          const T x1 = tau ? w1[l] : (l + 1 < NORD ? w1[l + 1] : T(0));
          a1 += __ldg(&I1[j * NORD + l]) * x1;
          a2 += __ldg(&I2[j * NORD + l]) * w2[l];
        }
        o1[j] = a1;
        o2[j] = a2;
      }
      const cpx<T> rc = {-rk.im, -rk.re};   // -i conj(rk)
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const T a1 = o1[2 * q], b1 = o1[2 * q + 1], a2 = o2[2 * q], b2 = o2[2 * q + 1];
        if (tau) {
          S[ws_at(P, Q, pen, q, p1)] = cmul(rk, cpx<T>{a2 - b2, a1 + b1});
          S[ws_at(P, Q, pen, q, p2)] = cmul(rc, cpx<T>{a1 - b1, a2 + b2});
        } else {
          S[ws_at(P, Q, pen, q, p1)] = cpx<T>{a1, b1};
          S[ws_at(P, Q, pen, q, p2)] = cmul(rk, cpx<T>{a2 - b2, a2 + b2});
        }
      }
    }
  }
  if (__syncthreads_or(nf) && threadIdx.x == 0 && P.nonfinite) atomicOr(P.nonfinite, 1);
}

// ------------------------------------------------------------ reconstruct

template <typename T, int NORD>
__global__ void __launch_bounds__(kLongThreads) long_reconstruct_kernel(LongParams P) {
  constexpr int Q = NORD / 2 + 1;
  const long long total = P.pencils * P.K;
  const cpx<T>* S = reinterpret_cast<const cpx<T>*>(P.S);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long pen, o, w;
    int e;
    split_item(P, t, P.K, pen, e);
    pencil_ow(P, pen, o, w);
    const int r = makhoul_inv(e, P.K);
    const T sg = (e & 1) ? T(-1) : T(1);
    T y[NORD];
    const cpx<T> x0 = S[ws_at(P, Q, pen, 0, r)];
    y[NORD - 1] = sg * x0.re + x0.im;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
      const cpx<T> x = S[ws_at(P, Q, pen, q, r)];
      const T ys = sg * x.re, yc = x.im;
      if (2 * q < NORD) {
        y[q - 1] = ys + yc;
        y[NORD - q - 1] = ys - yc;
      } else {
        y[q - 1] = ys;
      }
    }
    const long long m0 = (long long)NORD * e;
#pragma unroll
    for (int s = 0; s < NORD; ++s)
      if (!(s == NORD - 1 && e == P.K - 1)) store_out<T>(P, field_at(P, o, w, m0 + s), y[s]);
  }
}

}  // namespace

// ------------------------------------------------------------------- host

namespace {

// K = K1 K2 with K1 the 3-smooth "square root" (half the exponents, rounded down)
void long_split(int K, int* K1, int* K2) {
  int a = 0, b = 0, k = K;
  while (k % 2 == 0) { k /= 2; ++a; }
  while (k % 3 == 0) { k /= 3; ++b; }
  int k1 = 1;
  for (int i = 0; i < a / 2; ++i) k1 *= 2;
  for (int i = 0; i < b / 2; ++i) k1 *= 3;
  *K1 = k1;
  *K2 = K / k1;
}

// One FFT stage of length L.  Contiguous layout: count = sequences of length
// L per packed sequence, C of them per CTA (C | count).  Pencil-fastest
// layout (pf): count = lines of the stage, C adjacent pencils per CTA.
bool long_stage(int L, int count, int elem_bytes, bool cols, bool twiddle, bool pf, int Q, LongFft* F) {
  std::memset(F, 0, sizeof(*F));
  F->L = L;
  int r = L;
  while (r % 3 == 0) {
    F->radix[F->npass++] = 3;
    r /= 3;
  }
  while (r > 1) {
    const int R = r % 8 == 0 ? 8 : (r % 4 == 0 ? 4 : 2);
    if (r % R || F->npass >= kLongMaxPass) return false;
    F->radix[F->npass++] = R;
    r /= R;
  }
  F->pitch = L + 1;
  const long long budget = 96 * 1024;
  int C = 1;
  if (pf) {
    C = 16;
    while (C > 1 && 2LL * C * F->pitch * elem_bytes > budget) C /= 2;
  } else {
    while (C * 2 <= 16 && count % (C * 2) == 0 && 2LL * (C * 2) * F->pitch * elem_bytes <= budget) C *= 2;
  }
  if (2LL * C * F->pitch * elem_bytes > 200 * 1024) return false;
  F->C = C;
  F->cols = cols ? 1 : 0;
  F->twiddle = twiddle ? 1 : 0;
  F->pf = pf ? 1 : 0;
  F->Q = Q;
  if (pf) F->lines = count;
  else F->nblocks_per_seq = count / C;
  return true;
}

template <typename T, int NORD>
int long_launch_build(const LongParams& P, unsigned grid, cudaStream_t s) {
  long_build_kernel<T, NORD><<<grid, kLongThreads, 0, s>>>(P);
  return (int)cudaGetLastError();
}
template <typename T, int NORD>
int long_launch_reconstruct(const LongParams& P, unsigned grid, cudaStream_t s) {
  long_reconstruct_kernel<T, NORD><<<grid, kLongThreads, 0, s>>>(P);
  return (int)cudaGetLastError();
}
template <typename T, int NORD>
int long_launch_map(int mode, const LongParams& P, unsigned grid, cudaStream_t s) {
  if (mode == MODE_FWD) long_map_kernel<T, NORD, MODE_FWD><<<grid, kLongThreads, 0, s>>>(P);
  else if (mode == MODE_INV) long_map_kernel<T, NORD, MODE_INV><<<grid, kLongThreads, 0, s>>>(P);
  else long_map_kernel<T, NORD, MODE_FUSED><<<grid, kLongThreads, 0, s>>>(P);
  return (int)cudaGetLastError();
}

// what: 0 build, 1 reconstruct, 2 map
template <typename T>
int long_dispatch(int what, int n, int mode, const LongParams& P, unsigned grid, cudaStream_t s) {
#define FEMFFT_LONG_CASE(N)                                          \
  case N:                                                            \
    if (what == 0) return long_launch_build<T, N>(P, grid, s);       \
    if (what == 1) return long_launch_reconstruct<T, N>(P, grid, s); \
    return long_launch_map<T, N>(mode, P, grid, s);
  switch (n) {
    FEMFFT_LONG_CASE(1)
    FEMFFT_LONG_CASE(2)
    FEMFFT_LONG_CASE(3)
    FEMFFT_LONG_CASE(4)
    FEMFFT_LONG_CASE(5)
    FEMFFT_LONG_CASE(6)
    FEMFFT_LONG_CASE(7)
    FEMFFT_LONG_CASE(8)
    FEMFFT_LONG_CASE(9)
    default: return (int)cudaErrorInvalidValue;
  }
#undef FEMFFT_LONG_CASE
}

template <typename T>
int long_fft(const LongParams& P, const LongFft& F, long long nseq, cudaStream_t s) {
  const size_t smem = 2 * (size_t)F.C * F.pitch * sizeof(cpx<T>);
  const int e = ensure_dyn_smem((const void*)long_fft_kernel<T>, smem);
  if (e) return e;
  const long long grid = F.pf ? (long long)F.Q * F.lines * F.pblocks : nseq * F.nblocks_per_seq;
  if (grid > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
  long_fft_kernel<T><<<(unsigned)grid, kLongThreads, smem, s>>>(P, F);
  return (int)cudaGetLastError();
}

template <typename T>
int long_pass_t(fem_fft_plan p, int mode, int axis, long long outer, long long inner, const void* in, bool in_f64,
                void* out, bool out_f64, bool accum, int* nonfinite, cudaStream_t s) {
  const AxisHost& ax = p->ax[axis];
  const int n = ax.n, K = ax.K, M = ax.M, Q = n / 2 + 1;
  const DevTables& d = sizeof(T) == 8 ? p->t64[axis] : p->t32[axis];
  const bool pf = inner > 1;
  int K1, K2;
  long_split(K, &K1, &K2);
  // contiguous layout: count = the other factor (C columns / rows of one
  // sequence per CTA); pencil-fastest layout: count = lines of the stage
  LongFft cols_tw, rows, rows_tw, cols;
  const int eb = sizeof(cpx<T>);
  if (!long_stage(K1, K2, eb, true, true, pf, Q, &cols_tw) || !long_stage(K2, K1, eb, false, false, pf, Q, &rows) ||
      !long_stage(K2, K1, eb, false, true, pf, Q, &rows_tw) || !long_stage(K1, K2, eb, true, false, pf, Q, &cols)) {
    set_last_error("long pencil: no FFT schedule");
    return FEM_FFT_ERR_ARG;
  }
  // workspace: the packed sequences of a group of pencils (at most 256 MiB;
  // pencil-fastest groups are multiples of 16 pencils)
  const long long total = outer * inner;
  const size_t per_pencil = (size_t)Q * K * sizeof(cpx<T>);
  long long group = std::max<long long>(1, std::min<long long>(total, (256LL << 20) / (long long)per_pencil));
  if (pf) group = std::max<long long>(16, group / 16 * 16);
  const long long gpad = pf ? (group + 15) / 16 * 16 : group;
  const size_t need = (size_t)gpad * per_pencil;
  if (p->long_ws_bytes < need) {
    if (p->long_ws) {
      cudaStreamSynchronize(s);
      cudaFree(p->long_ws);
      p->long_ws = nullptr;
      p->long_ws_bytes = 0;
    }
    if (cudaMalloc(&p->long_ws, need) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("long pencil workspace: cudaMalloc failed");
      return FEM_FFT_ERR_OOM;
    }
    p->long_ws_bytes = need;
  }
  LongParams P;
  std::memset(&P, 0, sizeof(P));
  P.in = in;
  P.out = out;
  P.in_f64 = in_f64;
  P.out_f64 = out_f64;
  P.accum = accum;
  P.S = p->long_ws;
  P.inner = inner;
  P.pf = pf ? 1 : 0;
  P.K = K;
  P.K1 = K1;
  P.K2 = K2;
  P.M = M;
  P.n = n;
  P.tw = d.tw;
  P.rot = d.rot;
  P.fwd = p->use_fwdc ? d.fwdc : d.fwd;
  P.inv = d.inv;
  P.mu = d.mu;
  P.c = p->c;
  if (mode == MODE_FUSED) {   // the fused pass runs along axis 0: w indexes the later axes
    P.nother = p->N - 1;
    for (int j = 1; j < p->N; ++j) {
      P.Mo[j - 1] = p->M[j];
      P.mu_o[j - 1] = sizeof(T) == 8 ? p->t64[j].mu : p->t32[j].mu;
    }
  }
  P.nonfinite = nonfinite;
  int e = 0;
  for (long long g0 = 0; g0 < total && !e; g0 += group) {
    P.pencils = std::min(group, total - g0);
    P.first = g0;
    P.npad = pf ? (P.pencils + 15) / 16 * 16 : 0;
    for (LongFft* F : {&cols_tw, &rows, &rows_tw, &cols}) {
      F->npad = P.npad;
      F->pblocks = pf ? P.npad / F->C : 0;
    }
    const long long nseq = P.pencils * Q;
    const unsigned gridK = (unsigned)std::min<long long>((P.pencils * K + kLongThreads - 1) / kLongThreads, 152LL * 64);
    const unsigned gridH = (unsigned)std::min<long long>((P.pencils * (K / 2) + kLongThreads - 1) / kLongThreads, 152LL * 64);
    if (mode != MODE_INV) {
      if (!e) e = long_dispatch<T>(0, n, mode, P, gridK, s);
      if (!e) e = long_fft<T>(P, cols_tw, nseq, s);
      if (!e) e = long_fft<T>(P, rows, nseq, s);
    }
    if (!e) e = long_dispatch<T>(2, n, mode, P, gridH, s);
    if (mode != MODE_FWD) {
      if (!e) e = long_fft<T>(P, rows_tw, nseq, s);
      if (!e) e = long_fft<T>(P, cols, nseq, s);
      if (!e) e = long_dispatch<T>(1, n, mode, P, gridK, s);
    }
  }
  if (e) return cuda_fail((cudaError_t)e, "long pencil pass");
  return FEM_FFT_OK;
}

}  // namespace

int run_long_pass(fem_fft_plan p, int mode, int axis, long long outer, long long inner, const void* in,
                  bool in_f64, void* out, bool out_f64, bool accum, bool f64, int* nonfinite, cudaStream_t s) {
  if (mode == MODE_FUSED && axis != 0) {
    set_last_error("long pencils: the fused pass runs along axis 0");
    return FEM_FFT_ERR_ARG;
  }
  return f64 ? long_pass_t<double>(p, mode, axis, outer, inner, in, in_f64, out, out_f64, accum, nonfinite, s)
             : long_pass_t<float>(p, mode, axis, outer, inner, in, in_f64, out, out_f64, accum, nonfinite, s);
}

}  // namespace femfft
