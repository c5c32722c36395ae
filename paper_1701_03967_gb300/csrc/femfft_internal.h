// Internal structures shared by the host plan code and the CUDA kernels.
#pragma once
#include <cstdint>
#include <vector>

namespace femfft {

constexpr int kMaxN = 3;     // spatial dimensions
constexpr int kMaxOrder = 9; // element order n
constexpr int kFastMaxPass = 4;   // FFT passes of the register-radix pencil kernels

// Host-side 1D tables of one axis (all float64, computed in double-double and
// rounded once).  Spectral order of the M = nK-1 coefficients: sigma + 1 =
// n*k + slot, i.e. the n-1 bubble modes (k = 0, slot = l = 1..n-1) first,
// then for k = 1..K-1 the n modes l = 1..n at slots 0..n-1, with lambda
// ascending within each k.
struct AxisHost {
  int n = 0, K = 0, M = 0;
  double X = 1.0, a = 1.0, h = 1.0, s = 1.0;   // s = 4 / h^2
  std::vector<double> lam;     // [M] h-free eigenvalues (spectral order)
  std::vector<double> cnorm;   // [M] ||s||_C^2
  std::vector<double> mu;      // [M] a * s * lam
  std::vector<double> tw;      // [2K] exp(-2 pi i j / K), (re, im) pairs
  std::vector<double> rot;     // [2K] exp(-i pi k / (2K))
  std::vector<double> fwd;     // [K][n][2Q] per-k forward maps (Q = n/2+1); k = 0: bubble map
  std::vector<double> fwdc;    // [K][n][2Q] the same for the direct F_n-transform (mass product folded in)
  std::vector<double> inv;     // [K][2Q][n] per-k inverse maps; k = 0: bubble map
  std::vector<double> pvec;    // [K][n][n-1] p_k^(l) (k = 0: e^(l)), for tests
  std::vector<int> parity;     // [n-1] +1 even / -1 odd bubble eigenvector
  // tables of the register-radix passes (pencil_fast.cuh), for power-of-two
  // K in [16, 1024]; empty otherwise (fast_V == 0)
  int fast_V = 0, fast_npass = 0;
  int fast_radix[4] = {0, 0, 0, 0}, fast_lprod[4] = {0, 0, 0, 0}, fast_twofs[4] = {0, 0, 0, 0};
  std::vector<double> tw2;     // four-step twiddles [R0][K/R0], (re, im) pairs: exp(-2 pi i r i / K)
  std::vector<double> gmap;    // [2Q][n][K] inverse maps G_k[j][l] (the fwd table's transposed layout)
  std::vector<double> invn;    // [n][K] 1 / ||s_k^(l)||_C^2 (k = 0: 1/K, bubble modes l < n-1)
  std::vector<double> muk;     // [n][K] a s lambda of mode (k, l) (k = 0: bubble modes l < n-1)
};

// FFT schedule of the register-radix passes: V = 32 values per thread for
// K >= 512, else 16; passes of radix min(V, remaining).  False when K is not a
// power of two in [16, 1024].
bool fast_schedule(int K, int* V, int* npass, int* radix);
// Fill the fast_* tables of an axis whose base tables are computed (no-op
// when K is not eligible); fast_muk_update recomputes muk after a change of a.
void fast_tables(AxisHost* ax);
void fast_muk_update(AxisHost* ax);

// Precompute the tables of one axis.  Returns 0 or a negative status.
int precompute_axis(int n, int K, double X, double a, AxisHost* out);

// Generalized eigenpairs of the interior blocks of the reference element
// matrices, A_ii phi = nu C_ii phi (the bubble modes of Section 2), nu
// ascending, columns of phi ((n-1) x (n-1), row-major) C_ii-orthonormal.
// Returns 0 or a negative status; empty for n = 1.
int interior_eig(int n, std::vector<double>* nu, std::vector<double>* phi);

// Reference-element matrices rounded to double ((n+1)^2, row-major) and the
// row sums of C (those of A are exactly zero).
void reference_matrices(int n, std::vector<double>* A, std::vector<double>* C, std::vector<double>* Crow);

// Device view of one axis for one precision T (float or double).
struct AxisDev {
  int n, K, M;
  const void* tw;    // T2 [K]
  const void* rot;   // T2 [K]
  const void* fwd;   // T [K][n][2Q]
  const void* inv;   // T [K][2Q][n]
  const void* mu;    // T [M]
};

// Geometry of one pencil pass over a C-order array viewed as
// [outer][M][inner]: the pencils run along the middle index.
struct PassGeom {
  long long outer;   // slices before the axis (right-hand sides included)
  long long inner;   // product of the later axis sizes
  int M;             // pencil length
  int W;             // pencils per CTA (consecutive inner indices, or outer slices if inner == 1)
  long long tiles;   // number of CTAs
  long long tiles_inner;  // CTAs per outer slice (inner > 1)
};

// Extra data of the fused forward/divide/inverse pass on axis 0.
struct DivideDev {
  double c;               // zeroth-order coefficient
  int nother;             // number of other axes (0..2)
  long long Mo[2];        // their sizes (axis 1, axis 2)
  const void* mu_o[2];    // their a*s*lambda tables (T)
};

}  // namespace femfft
