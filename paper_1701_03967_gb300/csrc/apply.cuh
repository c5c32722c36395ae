// Matrix-free float64 application of the FEM operators along one axis.
//
// The 1D operators calA, calC of Section 2 are sums of the element blocks A, C
// ((n+1) x (n+1), Lagrange basis on [-1, 1]) over the K elements, with the two
// boundary vertices removed; their explicit rows are the node rows and the
// interior rows of the 1D system in Section 2.  The N-D operator of Section 4
// is a sum of Kronecker products of these, so L u (and the residual
// b - L u, and the bilinear forms lam^T (dL/da_i) u) are evaluated as a short
// chain of 1D applications along the axes, e.g. in 2D
//     w = (a_1 s_1 calA_1 + c calC_1) u (axis 1), t = a_2 s_2 calA_2 u (axis 2),
//     L u = calC_2 w + calC_1 t.
// In the float64 chains the stiffness factor of every term is applied to u
// itself and the mass factors afterwards: a float64 stiffness applied to an
// intermediate that carries rounding noise (such as calC_2 u) amplified
// that noise by ~4 h^-2 |A| and floored the refinement at ~6e-9 (2D, n = 9,
// K = 1024).  The double-float residual's shorter chain applies stiffness
// factors to double-float mass products; see operator_chain in api.cu.
// One thread computes the outputs of one element for all outputs of the
// launch; inputs are read through the read-only cache (along strided axes the
// threads of a warp cover consecutive positions of the contiguous axis).
// Every entry of the element matrices is applied in the even/odd form below.
#pragma once
#include <cuda_runtime.h>

#include "df64.cuh"
#include "kernels.h"

namespace femfft {

constexpr int kApplyThreads = 256;   // threads per CTA of the stand-alone apply kernel

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of up to 4 values, then one atomicAdd per value.  red: shared
// scratch of (blockDim.x / 32) * NV doubles.
template <int NV>
__device__ void block_accumulate(double (&v)[NV], double* dst, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) red[wid * NV + j] = v[j];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double x = lane < (int)(blockDim.x >> 5) ? red[lane * NV + j] : 0.0;
      x = warp_sum(x);
      if (lane == 0 && x != 0.0) atomicAdd(&dst[j], x);
    }
  }
}

// Even/odd element products.  A and C are bisymmetric (Section 2), so with
// the centre reference ub = (u_0 + u_n)/2 and d = u_e - ub 1 the product
// y = E d splits into half-size products of the symmetric sums
// s_q = d_q + d_{n-q} and the antisymmetric differences a_q = u_q - u_{n-q}:
//   y_q = Es'[q] . s + Ea'[q] . a,   y_{n-q} = Es'[q] . s - Ea'[q] . a   (q <= n/2),
// with Es'[q][j] = (E[q][j] + E[q][n-j]) / 2, Ea'[q][j] = (E[q][j] - E[q][n-j]) / 2
// (for even n the middle node enters Es' with E[q][n/2]).  The constant part
// is added back with the exact row sums: E u_e = E d + ub (E 1), and
// A 1 = 0 exactly (Section 2), so a stiffness term never multiplies the nodal
// values themselves -- for smooth u the sums s are O(h^2 u'') and the
// differences a are O(h u'), which keeps the float64 rounding of
// 4 h^-2 calA u far below the refinement target.  (Rounded A has row sums
// ~1e-14, not 0; using them would act as a spurious zeroth-order term and shift
// the refined solution by ~6e-9 at K = 1024, n = 9.)
//
// Layout of mats[t]: Es' (R x (P+1), the last column is the middle node of
// even n) followed by Ea' (R x P), R = n/2 + 1 rows q = 0..n/2, P = (n+1)/2
// pairs j < n/2.
//
// A block covers TW consecutive positions of the contiguous axis (w) times
// TE consecutive elements (TW * TE = kApplyThreads).  Each thread forms all
// n+1 local rows of its element; the vertex between elements e and e+1 adds
// row n of e and row 0 of e+1, exchanged through shared memory (the last
// element row of a tile recomputes its neighbour's row 0).
template <int NORD>
struct EO {
  static constexpr int N1 = NORD + 1;
  static constexpr int R = NORD / 2 + 1;
  static constexpr int P = (NORD + 1) / 2;
  static constexpr int SP = P + 1;     // columns of Es'
};

// NC: read through the read-only data cache; otherwise L2-coherent loads
// (fields written by other CTAs of the same launch).
template <bool NC>
__device__ __forceinline__ double ld_f64(const double* p) {
  if (NC) return __ldg(p);
  return __ldcg(p);
}

// local nodes of element e; gofs = 1: the field stores the boundary nodes
// too (fine index g at g + 1), so g = -1 and g = M are read, not zeroed
template <int NORD, bool NC>
__device__ __forceinline__ void load_elem(const double* x, long long line, long long inner, int e, int M,
                                          int gofs, double (&u)[NORD + 1]) {
#pragma unroll
  for (int q = 0; q <= NORD; ++q) {
    const int g = NORD * e + q - 1;
    u[q] = (g >= -gofs && g < M + gofs) ? ld_f64<NC>(&x[line + (long long)(g + gofs) * inner]) : 0.0;
  }
}

// y = E u for one element (all n+1 rows, or only row 0 when ROW0_ONLY)
template <int NORD, bool ROW0_ONLY>
__device__ __forceinline__ void elem_product(const double* Es, const double* Ea, const double* E1, bool has_e1,
                                             const double (&u)[NORD + 1], double (&y)[NORD + 1]) {
  using C = EO<NORD>;
  const double ub = 0.5 * (u[0] + u[NORD]);
  double sv[C::P + 1], av[C::P];
#pragma unroll
  for (int j = 0; j < C::P; ++j) {
    sv[j] = (u[j] + u[NORD - j]) - 2.0 * ub;
    av[j] = u[j] - u[NORD - j];
  }
  sv[C::P] = (NORD % 2 == 0) ? u[NORD / 2] - ub : 0.0;
  constexpr int NS = (NORD % 2 == 0) ? C::SP : C::P;   // the middle column exists for even n only
#pragma unroll
  for (int q = 0; q < C::R; ++q) {
    if (ROW0_ONLY && q > 0) break;
    double ts = 0.0, ta = 0.0;
#pragma unroll
    for (int j = 0; j < NS; ++j) ts = fma(Es[q * C::SP + j], sv[j], ts);
#pragma unroll
    for (int j = 0; j < C::P; ++j) ta = fma(Ea[q * C::P + j], av[j], ta);
    if (has_e1) {
      y[q] = fma(ub, E1[q], ts + ta);
      if (!ROW0_ONLY && NORD - q != q) y[NORD - q] = fma(ub, E1[NORD - q], ts - ta);
    } else {
      y[q] = ts + ta;
      if (!ROW0_ONLY && NORD - q != q) y[NORD - q] = ts - ta;
    }
  }
}

// Shared memory of one apply block (doubles unless noted): the even/odd
// halves Es', Ea' and row sums of every term, the row-0 exchange buffer and
// the reduction scratch.
template <int NORD, int NOUT, int NTHREADS>
struct ApplySmem {
  using C = EO<NORD>;
  double es[kApplyMaxTerms][C::R * C::SP];
  double ea[kApplyMaxTerms][C::R * C::P];
  double e1[kApplyMaxTerms][C::N1];
  double row0[NOUT][NTHREADS];
  double red[NTHREADS / 32][kApplyMaxOut];
  int has1[kApplyMaxTerms];
};

// Stage the element matrices of P's terms into shared memory (the caller
// synchronises before use).
template <int NORD, int NOUT, int NTHREADS>
__device__ __forceinline__ void apply_stage_mats(const ApplyParams& P, ApplySmem<NORD, NOUT, NTHREADS>& S) {
  using C = EO<NORD>;
  constexpr int N1 = C::N1;
  for (int t = 0; t < P.nterm; ++t) {
    for (int j = threadIdx.x; j < C::R * C::SP; j += blockDim.x) S.es[t][j] = P.mats[t][j];
    for (int j = threadIdx.x; j < C::R * C::P; j += blockDim.x) S.ea[t][j] = P.mats[t][C::R * C::SP + j];
    for (int r = threadIdx.x; r < N1; r += blockDim.x) S.e1[t][r] = P.rows1[t][r];
    if (threadIdx.x == 0) {
      int h = 0;
      for (int r = 0; r < N1; ++r) h |= P.rows1[t][r] != 0.0;
      S.has1[t] = h;
    }
  }
}

// Boundary-layer test of the Dirichlet correction (ApplyParams::bnd): true if
// one of element e's output rows (its interior rows and its right vertex)
// can be reached from the boundary of the operated axis -- e = 0, e = K - 1,
// and e = K - 2, whose right vertex takes row 0 of the last element -- or a
// stored index of another axis (extended fields: 0 .. M_j + 1) lies within
// one element of that axis's boundary.  Outside, every product of the chain
// is zero: each term of it applies one 1D operator per axis to data that is
// non-zero only at boundary nodes.
template <typename I>
__device__ __forceinline__ bool bnd_live_t(const ApplyParams& P, I o, I w, int e) {
  if (e == 0 || e >= P.K - 2) return true;
  for (int j = P.bnd_N - 1; j > P.bnd_axis; --j) {   // axes after the operated one: w, last axis fastest
    const I m = (I)P.bnd_M[j], n = (I)P.bnd_n[j];
    const I i = w % (m + 2);
    w /= m + 2;
    if (i <= n || i + n >= m + 1) return true;
  }
  for (int j = P.bnd_axis - 1; j >= 0; --j) {        // axes before it: o (right-hand side slowest)
    const I m = (I)P.bnd_M[j], n = (I)P.bnd_n[j];
    const I i = o % (m + 2);
    o /= m + 2;
    if (i <= n || i + n >= m + 1) return true;
  }
  return false;
}
// 32-bit divisions when the indices fit (they do for fields below 2^32 values)
__device__ __forceinline__ bool bnd_live(const ApplyParams& P, long long o, long long w, int e) {
  if (o < 0xffffffffLL && w < 0xffffffffLL) return bnd_live_t<unsigned>(P, (unsigned)o, (unsigned)w, e);
  return bnd_live_t<unsigned long long>(P, (unsigned long long)o, (unsigned long long)w, e);
}

// Block bx of an apply launch: TW consecutive positions of the contiguous
// axis times NTHREADS / TW consecutive elements of the operated axis.
template <int NORD, int NOUT, int NTHREADS, bool NC>
__device__ __forceinline__ void apply_block(const ApplyParams& P, int TW, long long bx,
                                            ApplySmem<NORD, NOUT, NTHREADS>& S) {
  using C = EO<NORD>;
  constexpr int N1 = C::N1;
  const int K = P.K;
  const int TE = NTHREADS / TW;
  // lines mode (inner == 1, TW > 1): TW lines of the contiguous axis per
  // block, threads along the elements of a line (as in apply_block_df)
  const bool lines = P.inner == 1 && TW > 1;
  const ApplyThread d = apply_decode(bx, (int)threadIdx.x, TW, NTHREADS, K, P.inner, P.outer, lines);
  const long long o = d.o, w = d.w;
  const int te = d.te, estep = d.estep, e = d.e;
  const bool valid = d.valid;
  const long long npos = d.npos;
  const long long Ms = P.M + 2 * P.gofs;   // stored extent of the operated axis
  const long long line = lines ? (valid ? w : 0) * Ms : o * Ms * P.inner + (valid ? w : 0);
  // in lines mode the line index is the outer index and no axis follows
  const bool live = valid && (!P.bnd || (lines ? bnd_live(P, w, 0, e) : bnd_live(P, o, w, e)));
  // a block outside every boundary layer has nothing to compute or store
  if (P.bnd && !__syncthreads_or(live)) return;

  double acc[NOUT][N1];
#pragma unroll
  for (int j = 0; j < NOUT; ++j)
#pragma unroll
    for (int q = 0; q < N1; ++q) acc[j][q] = 0.0;
  if (live) {
    for (int t = 0; t < P.nterm; ++t) {
      double u[N1], y[N1];
      load_elem<NORD, NC>(P.in[P.t_src[t]], line, P.inner, e, P.M, P.gofs, u);
      elem_product<NORD, false>(S.es[t], S.ea[t], S.e1[t], S.has1[t], u, y);
      const int d = P.t_dst[t];
#pragma unroll
      for (int j = 0; j < NOUT; ++j)
        if (j == d)
#pragma unroll
          for (int q = 0; q < N1; ++q) acc[j][q] += y[q];
    }
  }
#pragma unroll
  for (int j = 0; j < NOUT; ++j) S.row0[j][threadIdx.x] = acc[j][0];
  __syncthreads();

  double dotacc[kApplyMaxOut] = {0.0, 0.0, 0.0, 0.0};
  double rr = 0.0, bb = 0.0;
  if (live) {
    const bool has_node = e < K - 1;
    if (has_node) {
      if (te + 1 < TE) {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) acc[j][NORD] += S.row0[j][threadIdx.x + estep];
      } else {
        for (int t = 0; t < P.nterm; ++t) {
          double u[N1], y[N1];
          load_elem<NORD, NC>(P.in[P.t_src[t]], line, P.inner, e + 1, P.M, P.gofs, u);
          elem_product<NORD, true>(S.es[t], S.ea[t], S.e1[t], S.has1[t], u, y);
          const int d = P.t_dst[t];
#pragma unroll
          for (int j = 0; j < NOUT; ++j)
            if (j == d) acc[j][NORD] += y[0];
        }
      }
    }
    const int nrow = has_node ? NORD : NORD - 1;
#pragma unroll
    for (int r = 0; r < NORD; ++r) {
      if (r >= nrow) break;
      const long long off = line + (long long)(NORD * e + r + P.gofs) * P.inner;
      if (P.dotv) {
        const double lv = ld_f64<NC>(&P.dotv[off]);
#pragma unroll
        for (int j = 0; j < NOUT; ++j) dotacc[j] = fma(acc[j][r + 1], lv, dotacc[j]);
      } else {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
          if (j < P.nout) {
            double v = acc[j][r + 1];
            if (j == 0 && P.addend) v += NC ? P.addend[off] : __ldcg(&P.addend[off]);
            if (j == 0 && P.base) {
              double b = ld_f64<NC>(&P.base[off]);
              v = b - v;
              rr = fma(v, v, rr);
              bb = fma(b, b, bb);
            }
            if (j == 0 && P.out0_f32) P.out0_f32[off] = (float)v;
            else P.out[j][off] = v;
          }
        }
      }
    }
  }
  if (P.dotv) {
    block_accumulate<kApplyMaxOut>(dotacc, P.dots, &S.red[0][0]);
  } else if (P.norms) {
    double v2[2] = {rr, bb};
    block_accumulate<2>(v2, P.norms, &S.red[0][0]);
  }
}

// ---------------------------------------------------------- double-float
// The same even/odd element products in double-float arithmetic (about 48
// significant bits on the float pipes); used for the refinement residual.

template <int NORD, int NOUT, int NTHREADS>
struct ApplySmemDF {
  using C = EO<NORD>;
  df es[kApplyMaxTerms][C::R * C::SP];
  df ea[kApplyMaxTerms][C::R * C::P];
  df e1[kApplyMaxTerms][C::N1];
  df row0[NOUT][NTHREADS];
  double red[NTHREADS / 32][kApplyMaxOut];
  int has1[kApplyMaxTerms];
};

__device__ __forceinline__ df split_entry(double m) {
  const float hi = __double2float_rn(m);
  return {hi, __double2float_rn(m - (double)hi)};
}

template <int NORD, int NOUT, int NTHREADS>
__device__ __forceinline__ void apply_stage_mats_df(const ApplyParams& P, ApplySmemDF<NORD, NOUT, NTHREADS>& S) {
  using C = EO<NORD>;
  constexpr int N1 = C::N1;
  for (int t = 0; t < P.nterm; ++t) {
    for (int j = threadIdx.x; j < C::R * C::SP; j += blockDim.x) S.es[t][j] = split_entry(P.mats[t][j]);
    for (int j = threadIdx.x; j < C::R * C::P; j += blockDim.x) S.ea[t][j] = split_entry(P.mats[t][C::R * C::SP + j]);
    for (int r = threadIdx.x; r < N1; r += blockDim.x) S.e1[t][r] = split_entry(P.rows1[t][r]);
    if (threadIdx.x == 0) {
      int h = 0;
      for (int r = 0; r < N1; ++r) h |= P.rows1[t][r] != 0.0;
      S.has1[t] = h;
    }
  }
}

template <bool NC>
__device__ __forceinline__ float ld_f32(const float* p) {
  if (NC) return __ldg(p);
  return __ldcg(p);
}

// one value of an input field: a double-float field (two planes) or a
// float64 field split on load
template <bool NC>
__device__ __forceinline__ df ld_df(const double* x, bool is_df, long long plane, long long off) {
  if (is_df) {
    const float* f = reinterpret_cast<const float*>(x);
    return {ld_f32<NC>(f + off), ld_f32<NC>(f + plane + off)};
  }
  return split_f64(ld_f64<NC>(x + off));
}

// Input tiles of a double-float apply block, staged in shared memory before
// any arithmetic so that all of the block's loads are in flight together
// (the per-element loads of the unstaged form left the kernel waiting on
// memory latency).  Rows: fine indices g0 = n e0 - 1 .. n (e0 + TE + 1) - 1,
// i.e. the block's TE elements and the next element (whose row 0 the last
// element row recomputes); columns: the block's TW positions of the
// contiguous axis.  A slot holds the value as a (hi, lo) float pair: float64
// inputs are split once here, so the element products read every input the
// same way.
__host__ __device__ constexpr int apply_df_rows(int n, int TE) { return n * (TE + 1) + 1; }
inline size_t apply_df_tile_bytes(int n, int TW, int nthreads, int ninputs) {
  return (size_t)ninputs * apply_df_rows(n, nthreads / TW) * TW * 8;
}

constexpr int kStageBatch = 8;   // loads in flight per thread while staging

template <bool NC>
__device__ void stage_input_df(const double* x, bool is_df, long long plane, long long line0, long long inner,
                               int g0, int rows, int TW, int wvalid, int M, float2* tile) {
  const int total = rows * TW;
  const int tw_shift = __ffs(TW) - 1;   // TW is a power of two
  for (int i0 = threadIdx.x; i0 < total; i0 += kStageBatch * blockDim.x) {
    uint2 v[kStageBatch];
#pragma unroll
    for (int k = 0; k < kStageBatch; ++k) {
      const int i = i0 + k * blockDim.x;
      const int r = i >> tw_shift, c = i & (TW - 1);
      const int g = g0 + r;
      v[k] = make_uint2(0u, 0u);
      if (i < total && c < wvalid && g >= 0 && g < M) {
        const long long off = line0 + (long long)g * inner + c;
        if (is_df) {
          const float* f = reinterpret_cast<const float*>(x);
          v[k] = make_uint2(__float_as_uint(ld_f32<NC>(f + off)), __float_as_uint(ld_f32<NC>(f + plane + off)));
        } else {
          const unsigned long long bits = (unsigned long long)__double_as_longlong(ld_f64<NC>(x + off));
          v[k] = make_uint2((unsigned)bits, (unsigned)(bits >> 32));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kStageBatch; ++k) {
      const int i = i0 + k * blockDim.x;
      if (i < total) {
        df d;
        if (is_df) d = {__uint_as_float(v[k].x), __uint_as_float(v[k].y)};
        else d = split_f64(__longlong_as_double((long long)(((unsigned long long)v[k].y << 32) | v[k].x)));
        tile[i] = make_float2(d.hi, d.lo);
      }
    }
  }
}

// Lines mode (contiguous axis, several lines per block): column c of the
// tile is line w0 + c, rows g0 .. g0 + rows - 1 of it, stored [column][rows];
// consecutive threads load consecutive rows of one line.
template <bool NC>
__device__ void stage_lines_df(const double* x, bool is_df, long long plane, long long w0, int M, int g0, int rows,
                               int TW, int wvalid, float2* tile) {
  const int total = rows * TW;
  for (int i0 = threadIdx.x; i0 < total; i0 += kStageBatch * blockDim.x) {
    uint2 v[kStageBatch];
#pragma unroll
    for (int k = 0; k < kStageBatch; ++k) {
      const int i = i0 + k * blockDim.x;
      const int c = i / rows, r = i - c * rows;
      const int g = g0 + r;
      v[k] = make_uint2(0u, 0u);
      if (i < total && c < wvalid && g >= 0 && g < M) {
        const long long off = (w0 + c) * (long long)M + g;
        if (is_df) {
          const float* f = reinterpret_cast<const float*>(x);
          v[k] = make_uint2(__float_as_uint(ld_f32<NC>(f + off)), __float_as_uint(ld_f32<NC>(f + plane + off)));
        } else {
          const unsigned long long bits = (unsigned long long)__double_as_longlong(ld_f64<NC>(x + off));
          v[k] = make_uint2((unsigned)bits, (unsigned)(bits >> 32));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kStageBatch; ++k) {
      const int i = i0 + k * blockDim.x;
      if (i < total) {
        df d;
        if (is_df) d = {__uint_as_float(v[k].x), __uint_as_float(v[k].y)};
        else d = split_f64(__longlong_as_double((long long)(((unsigned long long)v[k].y << 32) | v[k].x)));
        tile[i] = make_float2(d.hi, d.lo);
      }
    }
  }
}

__device__ __forceinline__ df slot_df(float2 v) { return {v.x, v.y}; }

// y = E u for one element (all n+1 rows, or only row 0 when ROW0_ONLY) in
// the even/odd form of elem_product, reading u from a staged tile: u_q at
// col[q * TW].  The columns are streamed (runtime loop over the pairs j,
// n - j) and every row's compensated sum advances once per column, so the
// loop body stays small (the fully unrolled row-by-row form overflowed the
// instruction cache at n = 9) and the rows are independent chains.  Each
// row sees its terms in the order j = 0, 1, ...; column 0 of Es' multiplies
// s_0 = (u_0 + u_n) - 2 ub = 0 exactly and is skipped.  Every sum is
// renormalised: left unnormalised (lo parts of a few ulp of the operands, or
// of a row's partial sums) they are multiplied in float by the next product,
// which measured a floor of 1e-10 instead of ~1e-12 on the refined 2D n = 9
// solve.
template <int NORD, bool ROW0_ONLY>
__device__ __forceinline__ void elem_product_df(const df* Es, const df* Ea, const df* E1, bool has_e1,
                                                const float2* col, int TW, df (&y)[NORD + 1]) {
  using C = EO<NORD>;
  constexpr int RR = ROW0_ONLY ? 1 : C::R;
  const df u0 = slot_df(col[0]), un = slot_df(col[NORD * TW]);
  const df ub = df_scale2(df_add(u0, un), 0.5f);
  const df ub2 = df_scale2(ub, 2.0f);
  float ss[RR], cs[RR], sa[RR], ca[RR];
#pragma unroll
  for (int q = 0; q < RR; ++q) ss[q] = cs[q] = sa[q] = ca[q] = 0.0f;
  {
    const df av = df_sub(u0, un);
#pragma unroll
    for (int q = 0; q < RR; ++q) dot2_step(Ea[q * C::P], av, sa[q], ca[q]);
  }
#pragma unroll 1
  for (int j = 1; j < C::P; ++j) {
    const df uj = slot_df(col[j * TW]), unj = slot_df(col[(NORD - j) * TW]);
    const df sv = df_sub(df_add(uj, unj), ub2);
    const df av = df_sub(uj, unj);
#pragma unroll
    for (int q = 0; q < RR; ++q) {
      dot2_step(Es[q * C::SP + j], sv, ss[q], cs[q]);
      dot2_step(Ea[q * C::P + j], av, sa[q], ca[q]);
    }
  }
  if (NORD % 2 == 0) {   // the middle node (even n)
    const df sv = df_sub(slot_df(col[(NORD / 2) * TW]), ub);
#pragma unroll
    for (int q = 0; q < RR; ++q) dot2_step(Es[q * C::SP + C::P], sv, ss[q], cs[q]);
  }
#pragma unroll
  for (int q = 0; q < RR; ++q) {
    const df ts = {ss[q], cs[q]}, ta = {sa[q], ca[q]};
    if (has_e1) {
      y[q] = df_fma(ub, E1[q], df_add(ts, ta));
      if (!ROW0_ONLY && NORD - q != q) y[NORD - q] = df_fma(ub, E1[NORD - q], df_sub(ts, ta));
    } else {
      y[q] = df_add(ts, ta);
      if (!ROW0_ONLY && NORD - q != q) y[NORD - q] = df_sub(ts, ta);
    }
  }
}

// y = E u + F v for one element: two terms with their own matrices and
// inputs summed in the same compensated row sums (the even and odd halves
// of both products advance one set of accumulators), so that the sum costs
// no second set of n + 1 double-float rows.  Same column order per term as
// elem_product_df.
template <int NORD, bool ROW0_ONLY>
__device__ __forceinline__ void elem_product_df_sum2(const df* Es, const df* Ea, const df* E1, bool has_e1,
                                                     const float2* col, const df* Fs, const df* Fa, const df* F1,
                                                     bool has_f1, const float2* colf, int TW, df (&y)[NORD + 1]) {
  using C = EO<NORD>;
  constexpr int RR = ROW0_ONLY ? 1 : C::R;
  float ss[RR], cs[RR], sa[RR], ca[RR];
#pragma unroll
  for (int q = 0; q < RR; ++q) ss[q] = cs[q] = sa[q] = ca[q] = 0.0f;
  df ubt[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const float2* c = t == 0 ? col : colf;
    const df* Ms = t == 0 ? Es : Fs;
    const df* Ma = t == 0 ? Ea : Fa;
    const df u0 = slot_df(c[0]), un = slot_df(c[NORD * TW]);
    const df ub = df_scale2(df_add(u0, un), 0.5f);
    const df ub2 = df_scale2(ub, 2.0f);
    ubt[t] = ub;
    {
      const df av = df_sub(u0, un);
#pragma unroll
      for (int q = 0; q < RR; ++q) dot2_step(Ma[q * C::P], av, sa[q], ca[q]);
    }
#pragma unroll 1
    for (int j = 1; j < C::P; ++j) {
      const df uj = slot_df(c[j * TW]), unj = slot_df(c[(NORD - j) * TW]);
      const df sv = df_sub(df_add(uj, unj), ub2);
      const df av = df_sub(uj, unj);
#pragma unroll
      for (int q = 0; q < RR; ++q) {
        dot2_step(Ms[q * C::SP + j], sv, ss[q], cs[q]);
        dot2_step(Ma[q * C::P + j], av, sa[q], ca[q]);
      }
    }
    if (NORD % 2 == 0) {   // the middle node (even n)
      const df sv = df_sub(slot_df(c[(NORD / 2) * TW]), ub);
#pragma unroll
      for (int q = 0; q < RR; ++q) dot2_step(Ms[q * C::SP + C::P], sv, ss[q], cs[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < RR; ++q) {
    const df ts = {ss[q], cs[q]}, ta = {sa[q], ca[q]};
    df lo = df_add(ts, ta), hi = df_sub(ts, ta);
    if (has_e1) {
      lo = df_fma(ubt[0], E1[q], lo);
      hi = df_fma(ubt[0], E1[NORD - q], hi);
    }
    if (has_f1) {
      lo = df_fma(ubt[1], F1[q], lo);
      hi = df_fma(ubt[1], F1[NORD - q], hi);
    }
    y[q] = lo;
    if (!ROW0_ONLY && NORD - q != q) y[NORD - q] = hi;
  }
}

// Block bx of a double-float apply launch (same tiling as apply_block);
// tiles: shared memory for the staged inputs (apply_df_tile_bytes).
// LM: 0 the positions of the other axes per block, 1 lines mode (the caller
// has checked inner == 1 and TW > 1), 2 decided here (the batched kernel)
template <int NORD, int NOUT, int NTHREADS, bool NC, int LM = 2, bool SUMT = false>
__device__ __forceinline__ void apply_block_df(const ApplyParams& P, int TW, long long bx,
                                               ApplySmemDF<NORD, NOUT, NTHREADS>& S, float2* tiles) {
  static_assert(!SUMT || NOUT == 1, "summed terms use one accumulator");
  using C = EO<NORD>;
  constexpr int N1 = C::N1;
  const int K = P.K;
  const int TE = NTHREADS / TW;
  // Lines mode: on the contiguous axis (inner == 1) the host may put TW > 1
  // lines of TE elements into a block (TE about K), so that short lines do
  // not leave most threads without an element; threads then run along the
  // elements of a line and the tiles hold one column per line.
  const bool lines = LM == 2 ? (P.inner == 1 && TW > 1) : LM == 1;
  const ApplyThread d = apply_decode(bx, (int)threadIdx.x, TW, NTHREADS, K, P.inner, P.outer, lines);
  const long long npos = d.npos, et = d.et, o = d.o, w = d.w;
  const int tw = d.tw, te = d.te, estep = d.estep, e = d.e;
  const bool valid = d.valid;
  const long long w0 = d.wt * TW;
  const long long line = lines ? (valid ? w : 0) * (long long)P.M : o * (long long)P.M * P.inner + (valid ? w : 0);
  const long long plane = P.plane;
  const int rows = apply_df_rows(NORD, TE);
  const int g0 = NORD * (int)(et * TE) - 1;
  const int wvalid = (int)min((long long)TW, npos - w0);
  const int rstride = lines ? 1 : TW;      // tile distance between rows of one column
  const int cstride = lines ? rows : 1;    // and between columns
  // stage every input the block uses
  float2* tin[kApplyMaxIn];
  int nstaged = 0;
  for (int i = 0; i < kApplyMaxIn; ++i) {
    tin[i] = tiles + (size_t)nstaged * rows * TW;
    if (P.in[i]) {
      if (lines)
        stage_lines_df<NC>(P.in[i], P.in_df[i] != 0, plane, w0, P.M, g0, rows, TW, wvalid, tin[i]);
      else
        stage_input_df<NC>(P.in[i], P.in_df[i] != 0, plane, o * (long long)P.M * P.inner + w0, P.inner, g0, rows,
                           TW, wvalid, P.M, tin[i]);
      ++nstaged;
    }
  }
  __syncthreads();

  // term t writes output t (nterm == nout, checked on the host), so each
  // product lands in its accumulator directly
  df acc[NOUT][N1];
  if constexpr (SUMT) {
    const int off = NORD * te * rstride + tw * cstride;
    if (valid) {
      elem_product_df_sum2<NORD, false>(S.es[0], S.ea[0], S.e1[0], S.has1[0], tin[P.t_src[0]] + off, S.es[1],
                                        S.ea[1], S.e1[1], S.has1[1], tin[P.t_src[1]] + off, rstride, acc[0]);
    } else {
#pragma unroll
      for (int q = 0; q < N1; ++q) acc[0][q] = df{0.0f, 0.0f};
    }
  } else {
#pragma unroll
    for (int j = 0; j < NOUT; ++j) {
      if (valid && j < P.nterm) {
        elem_product_df<NORD, false>(S.es[j], S.ea[j], S.e1[j], S.has1[j],
                                     tin[P.t_src[j]] + NORD * te * rstride + tw * cstride, rstride, acc[j]);
      } else {
#pragma unroll
        for (int q = 0; q < N1; ++q) acc[j][q] = df{0.0f, 0.0f};
      }
    }
  }
  if (NOUT == 2 && P.sum_terms && valid) {   // both products into output 0
#pragma unroll
    for (int q = 0; q < N1; ++q) acc[0][q] = df_add(acc[0][q], acc[NOUT - 1][q]);
  }
#pragma unroll
  for (int j = 0; j < NOUT; ++j) S.row0[j][threadIdx.x] = acc[j][0];
  __syncthreads();
  // outputs this launch writes (one when the terms are summed)
  constexpr bool kOne = NOUT == 1;
  const bool one_out = kOne || P.sum_terms;

  float rr = 0.0f, bb = 0.0f;
  if (valid) {
    const bool has_node = e < K - 1;
    if (has_node) {
      if (te + 1 < TE) {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) acc[j][NORD] = df_add(acc[j][NORD], S.row0[j][threadIdx.x + estep]);
      } else if constexpr (SUMT) {
        const int off = NORD * (te + 1) * rstride + tw * cstride;
        df y[N1];
        elem_product_df_sum2<NORD, true>(S.es[0], S.ea[0], S.e1[0], S.has1[0], tin[P.t_src[0]] + off, S.es[1],
                                         S.ea[1], S.e1[1], S.has1[1], tin[P.t_src[1]] + off, rstride, y);
        acc[0][NORD] = df_add(acc[0][NORD], y[0]);
      } else {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
          if (j < P.nterm) {
            df y[N1];
            elem_product_df<NORD, true>(S.es[j], S.ea[j], S.e1[j], S.has1[j],
                                        tin[P.t_src[j]] + NORD * (te + 1) * rstride + tw * cstride, rstride, y);
            if (NOUT == 2 && P.sum_terms) acc[0][NORD] = df_add(acc[0][NORD], y[0]);
            else acc[j][NORD] = df_add(acc[j][NORD], y[0]);
          }
        }
      }
    }
  }
  // Plain double-float outputs of a block narrower than a warp (TW < 32:
  // the contiguous axis has TW = 1) leave through the input tiles, which
  // are free now: written per element, stored row by row so that a warp's
  // stores are contiguous (a thread's own rows are TW * inner apart).
  const int orows = NORD * TE;
  const int tile_cap = P.tile_cap > nstaged ? P.tile_cap : nstaged;
  const bool stage_out = TW < 32 && !P.base && !P.addend && !P.out0_f32 && P.nout * orows <= tile_cap * rows;
  if (stage_out) {
    __syncthreads();   // every staged input has been read
    if (valid) {
      const int nrow = e < K - 1 ? NORD : NORD - 1;
#pragma unroll
      for (int r = 0; r < NORD; ++r) {
        if (r >= nrow) break;
#pragma unroll
        for (int j = 0; j < NOUT; ++j)
          if (j < P.nout)
            tiles[(size_t)j * orows * TW + (size_t)(NORD * te + r) * rstride + (size_t)tw * (lines ? orows : 1)] =
                make_float2(acc[j][r + 1].hi, acc[j][r + 1].lo);
      }
    }
    __syncthreads();
    const int g_first = NORD * (int)(et * TE);
    const int rows_out = min(orows, P.M - g_first);
    const int tw_shift = __ffs(TW) - 1;
    const long long base_off = o * (long long)P.M * P.inner + (long long)g_first * P.inner + w0;
    auto put = [&](int i, long long off) {
#pragma unroll
      for (int j = 0; j < NOUT; ++j)
        if (j < P.nout) {
          const float2 v = tiles[(size_t)j * orows * TW + i];
          float* f = reinterpret_cast<float*>(P.out[j]);
          f[off] = v.x;
          f[plane + off] = v.y;
        }
    };
    if (lines) {   // tile index i = c * orows + rho
      for (int i = threadIdx.x; i < orows * TW; i += blockDim.x) {
        const int c = i / orows, rho = i - c * orows;
        if (c < wvalid && rho < rows_out) put(i, (w0 + c) * (long long)P.M + g_first + rho);
      }
    } else {       // tile index i = rho * TW + c
      for (int i = threadIdx.x; i < rows_out * TW; i += blockDim.x) {
        const int rho = i >> tw_shift, c = i & (TW - 1);
        if (c < wvalid) put(i, base_off + (long long)rho * P.inner + c);
      }
    }
    return;
  }
  if (valid) {
    const bool has_node = e < K - 1;
    const int nrow = has_node ? NORD : NORD - 1;
    // every row's addend and base values are loaded before the first store:
    // issued inside the store loop, the float loads of a row could not pass
    // the float stores of the rows before it and each row waited on memory
    if (one_out && P.addend) {
      float2 ad[NORD];
#pragma unroll
      for (int r = 0; r < NORD; ++r) {
        const long long off = line + (long long)(NORD * e + min(r, nrow - 1)) * P.inner;
        const float* a = reinterpret_cast<const float*>(P.addend);
        ad[r] = make_float2(ld_f32<NC>(a + off), ld_f32<NC>(a + plane + off));
      }
#pragma unroll
      for (int r = 0; r < NORD; ++r) acc[0][r + 1] = df_add(acc[0][r + 1], df{ad[r].x, ad[r].y});
    }
    double bv[NORD];
    if (one_out && P.base) {
#pragma unroll
      for (int r = 0; r < NORD; ++r)
        bv[r] = ld_f64<NC>(&P.base[line + (long long)(NORD * e + min(r, nrow - 1)) * P.inner]);
    }
#pragma unroll
    for (int r = 0; r < NORD; ++r) {
      if (r >= nrow) break;
      const long long off = line + (long long)(NORD * e + r) * P.inner;
#pragma unroll
      for (int j = 0; j < NOUT; ++j) {
        if (j < P.nout) {
          df v = acc[j][r + 1];
          if (one_out && P.base) {
            const df b = split_f64(bv[r]);
            const float rv = df_to_float(df_sub(b, v));
            rr = fmaf(rv, rv, rr);
            bb = fmaf(b.hi, b.hi, bb);
            P.out0_f32[off] = rv;
          } else if (j == 0 && P.out0_f32) {
            P.out0_f32[off] = df_to_float(v);
          } else {
            float* f = reinterpret_cast<float*>(P.out[j]);
            f[off] = v.hi;
            f[plane + off] = v.lo;
          }
        }
      }
    }
  }
  if (P.norms) {
    double v2[2] = {(double)rr, (double)bb};
    block_accumulate<2>(v2, P.norms, &S.red[0][0]);
  }
}

}  // namespace femfft
