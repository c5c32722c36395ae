// Device code of algorithm (b) of Section 4 along axis 0: after the direct
// FC_n-transforms in the later axes, every position w of those axes carries an independent
// 1D problem [alpha calA + beta_w calC] v = y in x_1 (alpha = a_1 4 h_1^-2,
// beta_w = c + sum_{i>=2} a_i 4 h_i^-2 lambda_i), symmetric positive definite
// with half-bandwidth n.
//
// It is solved by static condensation, which is the banded factorisation
// ordered element interiors first:
//  1. per element (parallel): the interior block E_ii = alpha A_ii + beta C_ii
//     is inverted through the generalized eigenvectors of (A_ii, C_ii) (the
//     bubble modes of Section 2): E_ii^-1 = Phi diag(r) Phi^T with
//     r_m = 1 / (alpha nu_m + beta); z = E_ii^-1 y_i replaces the interiors,
//     the condensed right-hand side y_v - E_bi z is formed for the vertices;
//  2. per 1D problem (parallel over w): the vertex system is symmetric
//     tridiagonal with constant coefficients from the element Schur
//     complement S = E_bb - E_bi E_ii^-1 E_ib: tridiag(off, D, off) =
//     2 delta I - off T2, T2 = tridiag(-1, 2, -1), off = S_01, delta its row
//     sum.  For off < 0 (stiffness-dominated) it is solved as
//     (-off)(sigma I + T2) with sigma = 2 delta / (-off), by elimination
//     whose pivots 1 + e_j, e_1 = 1 + sigma, e_j = sigma + e_{j-1} / (1 + e_{j-1})
//     involve no cancellation (the plain form subtracts numbers that agree to
//     many digits for the lowest modes, where the system is nearly the
//     singular T2); for off >= 0 (mass-dominated, strongly diagonally
//     dominant) by plain elimination.  No pivoting: the matrices are
//     symmetric positive definite;
//  3. per element (parallel): interiors v_i = z - E_ii^-1 E_ib v_b.
// Every thread writes only its own element's slots; the right-vertex
// contribution of element e goes to a scratch row and is added by the
// vertex solve, so the result does not depend on thread timing.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace femfft {

constexpr int kBandThreads = 256;

// Field loads.  Every phase writes the field it reads, so no load goes
// through the read-only cache.  L2: cached in L2 only, for the batched kernel,
// which reads what other CTAs of the same launch wrote in earlier steps (an
// SM's L1 is not coherent with the other SMs' stores).
template <bool L2, typename T>
__device__ __forceinline__ T band_ld(const T* p) {
  if (L2) return __ldcg(p);
  return *p;
}

template <typename T>
struct ElemData;
template <>
struct ElemData<double> {
  __device__ static double phi(const BandParams& P, int i) { return P.phi[i]; }
  __device__ static double pta(const BandParams& P, int l, int b) { return P.pta[l][b]; }
  __device__ static double ptc(const BandParams& P, int l, int b) { return P.ptc[l][b]; }
  __device__ static double abi(const BandParams& P, int b, int m) { return P.abi[b][m]; }
  __device__ static double cbi(const BandParams& P, int b, int m) { return P.cbi[b][m]; }
};
template <>
struct ElemData<float> {
  __device__ static float phi(const BandParams& P, int i) { return P.phif[i]; }
  __device__ static float pta(const BandParams& P, int l, int b) { return P.ptaf[l][b]; }
  __device__ static float ptc(const BandParams& P, int l, int b) { return P.ptcf[l][b]; }
  __device__ static float abi(const BandParams& P, int b, int m) { return P.abif[b][m]; }
  __device__ static float cbi(const BandParams& P, int b, int m) { return P.cbif[b][m]; }
};

// Element blocks of the condensation and back substitution: TW positions of
// the contiguous axis times kBandThreads / TW elements.
__host__ __device__ inline long long band_elem_blocks(const BandParams& P, int TW) {
  const int TE = kBandThreads / TW;
  return P.outer * ((P.inner + TW - 1) / TW) * ((P.K + TE - 1) / TE);
}
__host__ __device__ inline int band_tw(long long inner) {
  int TW = 1;
  while (TW * 2 <= 32 && TW * 2 <= inner) TW *= 2;
  return TW;
}
// Blocks of the vertex solve: one thread per position.
__host__ __device__ inline long long band_vertex_blocks(const BandParams& P) {
  return (P.outer * P.inner + kBandThreads - 1) / kBandThreads;
}

// block bx -> (outer o, element e, position w); false if out of range
__device__ __forceinline__ bool band_elem(const BandParams& P, int TW, long long bx, long long& o, int& e,
                                          long long& w) {
  const int TE = kBandThreads / TW;
  const long long wtiles = (P.inner + TW - 1) / TW;
  const long long etiles = (P.K + TE - 1) / TE;
  const long long et = bx % etiles;
  bx /= etiles;
  const long long wt = bx % wtiles;
  o = bx / wtiles;
  w = wt * TW + threadIdx.x % TW;
  e = (int)(et * TE + threadIdx.x / TW);
  return w < P.inner && e < P.K;
}

template <typename T, int NORD, bool L2>
__device__ __forceinline__ void band_condense_block(const BandParams& P, int TW, long long bx) {
  constexpr int NI = NORD - 1, NI1 = NI > 0 ? NI : 1;
  using D = ElemData<T>;
  long long o, w;
  int e;
  if (!band_elem(P, TW, bx, o, e, w)) return;
  T* f = reinterpret_cast<T*>(P.f);
  T* scr = reinterpret_cast<T*>(P.scr);
  const long long line = o * (long long)P.M * P.inner + w;
  const long long npen = P.outer * P.inner, pen = o * P.inner + w;
  const T* tab = reinterpret_cast<const T*>(P.tab) + w * (NORD + 2);
  const T beta = tab[0], alpha = T(P.alpha);
  T gl = T(0), gr = T(0);
  if (NI > 0) {
    T y[NI1], s[NI1];
#pragma unroll
    for (int m = 0; m < NI; ++m) y[m] = band_ld<L2>(&f[line + (long long)(NORD * e + m) * P.inner]);
#pragma unroll
    for (int l = 0; l < NI; ++l) {
      T acc = T(0);
#pragma unroll
      for (int i = 0; i < NI; ++i) acc = fma(D::phi(P, i * NI + l), y[i], acc);
      s[l] = acc * tab[1 + l];
    }
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      T z = T(0);
#pragma unroll
      for (int l = 0; l < NI; ++l) z = fma(D::phi(P, i * NI + l), s[l], z);
      f[line + (long long)(NORD * e + i) * P.inner] = z;
      gl = fma(alpha * D::abi(P, 0, i) + beta * D::cbi(P, 0, i), z, gl);
      gr = fma(alpha * D::abi(P, 1, i) + beta * D::cbi(P, 1, i), z, gr);
    }
  }
  if (e >= 1) {
    const long long v = line + (long long)(NORD * e - 1) * P.inner;   // left vertex of element e
    f[v] = band_ld<L2>(&f[v]) - gl;
  }
  if (e <= P.K - 2) scr[(long long)e * npen + pen] = -gr;
}

template <typename T>
__device__ __forceinline__ T band_recip(T d);
template <>
__device__ __forceinline__ float band_recip(float d) { return 1.0f / d; }
template <>
__device__ __forceinline__ double band_recip(double d) { return 1.0 / d; }

template <typename T, int NORD, bool L2>
__device__ __forceinline__ void band_vertex_block(const BandParams& P, long long bx) {
  const long long npen = P.outer * P.inner;
  const long long pen = bx * kBandThreads + threadIdx.x;
  if (pen >= npen) return;
  const long long o = pen / P.inner, w = pen - o * P.inner;
  T* f = reinterpret_cast<T*>(P.f);
  T* scr = reinterpret_cast<T*>(P.scr);
  const long long line = o * (long long)P.M * P.inner + w;
  const T* tab = reinterpret_cast<const T*>(P.tab) + w * (NORD + 2);
  const T sd = tab[NORD], off = tab[NORD + 1];
  const bool stiff = off < T(0);
  // stiff: (sigma I + T2) v = g / (-off), eliminated with sub-diagonal -1;
  // else: tridiag(off, D, off) v = g, eliminated with sub-diagonal off
  const T scale = stiff ? band_recip<T>(-off) : T(1);
  const T sub = stiff ? T(-1) : off;
  const int nv = P.K - 1;   // vertices j = 1..K-1 at fine index n j - 1
  constexpr int B = 8;      // loads issued ahead of the elimination
  T e = T(0), cp = T(0), dp = T(0);
  for (int j0 = 1; j0 <= nv; j0 += B) {
    T g[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int j = j0 + k;
      g[k] = T(0);
      if (j <= nv)
        g[k] = band_ld<L2>(&f[line + (long long)(NORD * j - 1) * P.inner]) +
               band_ld<L2>(&scr[(long long)(j - 1) * npen + pen]);
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int j = j0 + k;
      if (j <= nv) {
        T inv;
        if (stiff) {
          e = (j == 1) ? T(1) + sd : sd + e * cp;   // pivot 1 + e_j; cp holds 1 / (1 + e_{j-1})
          inv = band_recip<T>(T(1) + e);
        } else {
          inv = band_recip<T>(sd - off * cp);       // cp holds off / pivot_{j-1}
        }
        dp = (g[k] * scale - sub * dp) * inv;
        cp = stiff ? inv : off * inv;
        scr[(long long)(j - 1) * npen + pen] = cp;
        f[line + (long long)(NORD * j - 1) * P.inner] = dp;
      }
    }
  }
  // back substitution v_j = dp_j - c_j v_{j+1}, c_j = super / pivot_j
  const T sup = stiff ? T(-1) : T(1);
  T vnext = T(0);
  for (int j0 = nv; j0 >= 1; j0 -= B) {
    T d[B], c[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int j = j0 - k;
      d[k] = c[k] = T(0);
      if (j >= 1) {
        d[k] = band_ld<L2>(&f[line + (long long)(NORD * j - 1) * P.inner]);
        c[k] = band_ld<L2>(&scr[(long long)(j - 1) * npen + pen]);
      }
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int j = j0 - k;
      if (j >= 1) {
        vnext = d[k] - sup * c[k] * vnext;
        f[line + (long long)(NORD * j - 1) * P.inner] = vnext;
      }
    }
  }
}

template <typename T, int NORD, bool L2>
__device__ __forceinline__ void band_back_block(const BandParams& P, int TW, long long bx) {
  constexpr int NI = NORD - 1, NI1 = NI > 0 ? NI : 1;
  using D = ElemData<T>;
  if (NI == 0) return;
  long long o, w;
  int e;
  if (!band_elem(P, TW, bx, o, e, w)) return;
  T* f = reinterpret_cast<T*>(P.f);
  const long long line = o * (long long)P.M * P.inner + w;
  const T* tab = reinterpret_cast<const T*>(P.tab) + w * (NORD + 2);
  const T beta = tab[0], alpha = T(P.alpha);
  const T vl = e >= 1 ? band_ld<L2>(&f[line + (long long)(NORD * e - 1) * P.inner]) : T(0);
  const T vr = e <= P.K - 2 ? band_ld<L2>(&f[line + (long long)(NORD * e + NORD - 1) * P.inner]) : T(0);
  T t[NI1];
#pragma unroll
  for (int l = 0; l < NI; ++l) {
    const T el = alpha * D::pta(P, l, 0) + beta * D::ptc(P, l, 0);
    const T er = alpha * D::pta(P, l, 1) + beta * D::ptc(P, l, 1);
    t[l] = fma(el, vl, er * vr) * tab[1 + l];
  }
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const long long g = line + (long long)(NORD * e + i) * P.inner;
    T acc = band_ld<L2>(&f[g]);
#pragma unroll
    for (int l = 0; l < NI; ++l) acc = fma(-D::phi(P, i * NI + l), t[l], acc);
    f[g] = acc;
  }
}

}  // namespace femfft
