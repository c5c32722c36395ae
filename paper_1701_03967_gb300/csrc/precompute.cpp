// Plan precompute: reference-element matrices, 1D eigenpairs and the per-axis
// transform tables, all in double-double arithmetic and rounded once to
// double.  Host code only; compile with -ffp-contract=off (see dd.h).
//
// Paper passages (Zlotnik & Zlotnik, arXiv:1701.03967):
//  * Section 2: local stiffness/mass matrices A, C on [-1, 1] with the
//    Lagrange basis at -1 + 2k/n; their 3x3 block (bisymmetric) form; the
//    interior element eigenproblem A~ e = lambda C~ e with C~ e.e = 1 and
//    even/odd eigenvectors (Lemma 1).
//  * Section 3, Theorem 1: the eigenvalues lambda_k^(l) (n per k = 1..K-1)
//    and the vectors p_k^(l) of the eigenvectors s_k^(l) (node values
//    sin(pi k j / K), interiors p sin(pi k (j-1)/K) + flip(p) sin(pi k j / K)).
//    Here they are obtained as the n eigenpairs of the restriction of the
//    pencil (calA, calC) to the n-dimensional space spanned by s_k^(1..n):
//    for a vector z = (v, p) the Rayleigh quotient of s(z) is
//    z^T A_theta z / z^T C_theta z with A_theta = A00 + theta (AJ)00 (leading
//    n x n block of A and of A times the flip J), likewise C_theta; the
//    eigenvector scaled to v = 1 gives p_k^(l), and ||s_k^(l)||_C^2 =
//    K z^T C_theta z (the norm formula of Theorem 2, item 2, in matrix form).
//  * Section 3, Theorem 2: the fast transforms.  The per-k maps stored here
//    implement items 1 and 2 with the node and interior parts written as
//    half-sample sine/cosine sums (see pencil.cuh for the derivation).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "dd.h"
#include "femfft_internal.h"

namespace femfft {

// --------------------------------------------------------------- sin / cos

static void taylor_sincos(const dd& x, dd* s, dd* c) {
  // |x| <= pi/4: terms fall below 1e-34 well before k = 40
  dd x2 = x * x;
  dd term = x, sum_s = x;
  for (int k = 1; k < 40; ++k) {
    term = term * x2 / dd(double((2 * k) * (2 * k + 1)));
    term = -term;
    sum_s += term;
    if (std::fabs(term.hi) < 1e-34) break;
  }
  dd termc(1.0), sum_c(1.0);
  for (int k = 1; k < 40; ++k) {
    termc = termc * x2 / dd(double((2 * k - 1) * (2 * k)));
    termc = -termc;
    sum_c += termc;
    if (std::fabs(termc.hi) < 1e-34) break;
  }
  *s = sum_s;
  *c = sum_c;
}

void dd_sincospi_frac(long long num, long long den, dd* s, dd* c) {
  // angle = pi * num / den, reduced exactly: r = num mod 2den in [0, 2den)
  long long twod = 2 * den;
  long long r = num % twod;
  if (r < 0) r += twod;
  long long o = (4 * r) / den;          // octant 0..7
  long long q = o / 2, h = o % 2;
  dd sb, cb;
  if (h == 0) {
    // beta = pi (4r - o den) / (4 den) in [0, pi/4)
    dd y = dd_pi() * dd(double(4 * r - o * den)) / dd(double(4 * den));
    taylor_sincos(y, &sb, &cb);
  } else {
    // beta = pi/2 - y', y' = pi ((o+1) den - 4r) / (4 den) in (0, pi/4]
    dd y = dd_pi() * dd(double((o + 1) * den - 4 * r)) / dd(double(4 * den));
    dd sy, cy;
    taylor_sincos(y, &sy, &cy);
    sb = cy;
    cb = sy;
  }
  switch (q) {
    case 0: *s = sb; *c = cb; break;
    case 1: *s = cb; *c = -sb; break;
    case 2: *s = -sb; *c = -cb; break;
    default: *s = -cb; *c = sb; break;
  }
}

// ------------------------------------------------- reference element (Sec. 2)

static void gauss_legendre(int G, std::vector<dd>* x, std::vector<dd>* w) {
  x->assign(G, dd(0.0));
  w->assign(G, dd(0.0));
  for (int i = 0; i < G; ++i) {
    dd z(std::cos(M_PI * (i + 0.75) / (G + 0.5)));
    dd dp;
    for (int it = 0; it < 100; ++it) {
      dd p0(1.0), p1 = z;
      for (int k = 2; k <= G; ++k) {
        dd p2 = (dd(double(2 * k - 1)) * z * p1 - dd(double(k - 1)) * p0) / dd(double(k));
        p0 = p1;
        p1 = p2;
      }
      // P_G(z) = p1, P_{G-1}(z) = p0; P'_G = G (z P_G - P_{G-1}) / (z^2 - 1)
      dp = dd(double(G)) * (z * p1 - p0) / (z * z - dd(1.0));
      dd dz = p1 / dp;
      z = z - dz;
      if (std::fabs(dz.hi) < 1e-33) break;
    }
    (*x)[i] = z;
    (*w)[i] = dd(2.0) / ((dd(1.0) - z * z) * dp * dp);
  }
}

// A_kl = int e_k' e_l', C_kl = int e_k e_l on [-1, 1] (n+1 Gauss points are
// exact for the degree-2n integrands), Lagrange basis at -1 + 2k/n.
static void reference_matrices_dd(int n, std::vector<dd>* A, std::vector<dd>* C) {
  int G = n + 1;
  std::vector<dd> xg, wg;
  gauss_legendre(G, &xg, &wg);
  std::vector<dd> nodes(n + 1);
  for (int k = 0; k <= n; ++k) nodes[k] = dd(-1.0) + dd(double(2 * k)) / dd(double(n));
  std::vector<dd> val((n + 1) * G), der((n + 1) * G);
  for (int l = 0; l <= n; ++l) {
    for (int g = 0; g < G; ++g) {
      dd prod(1.0), dsum(0.0);
      for (int m = 0; m <= n; ++m) {
        if (m == l) continue;
        dd f = (xg[g] - nodes[m]) / (nodes[l] - nodes[m]);
        // derivative of the product by the product rule
        dd dterm = dd(1.0) / (nodes[l] - nodes[m]);
        for (int m2 = 0; m2 <= n; ++m2) {
          if (m2 == l || m2 == m) continue;
          dterm = dterm * (xg[g] - nodes[m2]) / (nodes[l] - nodes[m2]);
        }
        dsum += dterm;
        prod = prod * f;
      }
      val[l * G + g] = prod;
      der[l * G + g] = dsum;
    }
  }
  std::vector<dd> Araw((n + 1) * (n + 1)), Craw((n + 1) * (n + 1));
  for (int k = 0; k <= n; ++k)
    for (int l = 0; l <= n; ++l) {
      dd sa(0.0), sc(0.0);
      for (int g = 0; g < G; ++g) {
        sa += wg[g] * der[k * G + g] * der[l * G + g];
        sc += wg[g] * val[k * G + g] * val[l * G + g];
      }
      Araw[k * (n + 1) + l] = sa;
      Craw[k * (n + 1) + l] = sc;
    }
  // A and C are symmetric and bisymmetric (Section 2); average the four
  // equivalent entries so that the rounded matrices keep both symmetries
  // exactly (the even/odd element products rely on it)
  A->assign((n + 1) * (n + 1), dd(0.0));
  C->assign((n + 1) * (n + 1), dd(0.0));
  for (int k = 0; k <= n; ++k)
    for (int l = 0; l <= n; ++l) {
      const int i0 = k * (n + 1) + l, i1 = l * (n + 1) + k, i2 = (n - k) * (n + 1) + (n - l),
                i3 = (n - l) * (n + 1) + (n - k);
      (*A)[i0] = (Araw[i0] + Araw[i1] + Araw[i2] + Araw[i3]) * dd(0.25);
      (*C)[i0] = (Craw[i0] + Craw[i1] + Craw[i2] + Craw[i3]) * dd(0.25);
    }
}

void reference_matrices(int n, std::vector<double>* A, std::vector<double>* C, std::vector<double>* Crow) {
  std::vector<dd> Ad, Cd;
  reference_matrices_dd(n, &Ad, &Cd);
  A->resize(Ad.size());
  C->resize(Cd.size());
  for (size_t i = 0; i < Ad.size(); ++i) {
    (*A)[i] = Ad[i].to_double();
    (*C)[i] = Cd[i].to_double();
  }
  if (Crow) {
    // row sums of C in double-double (those of A are exactly zero)
    Crow->assign(n + 1, 0.0);
    for (int r = 0; r <= n; ++r) {
      dd acc(0.0);
      for (int q = 0; q <= n; ++q) acc += Cd[r * (n + 1) + q];
      (*Crow)[r] = acc.to_double();
    }
  }
}

// ------------------------------------------- symmetric-definite eigenproblem

// A x = lambda B x, B SPD, m x m row-major; lambda ascending, columns of X
// B-orthonormal.  Cholesky reduction and cyclic Jacobi, all in dd.
static int sym_def_eig(int m, const std::vector<dd>& A, const std::vector<dd>& B,
                       std::vector<dd>* lam, std::vector<dd>* X) {
  std::vector<dd> L(m * m, dd(0.0));
  for (int j = 0; j < m; ++j) {
    dd d = B[j * m + j];
    for (int k = 0; k < j; ++k) d -= L[j * m + k] * L[j * m + k];
    if (d.hi <= 0.0) return -1;
    dd ljj = dd_sqrt(d);
    L[j * m + j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      dd s = B[i * m + j];
      for (int k = 0; k < j; ++k) s -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = s / ljj;
    }
  }
  // Y = L^{-1} A, S = Y L^{-T}
  std::vector<dd> Y(m * m), S(m * m);
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < m; ++i) {
      dd s = A[i * m + c];
      for (int k = 0; k < i; ++k) s -= L[i * m + k] * Y[k * m + c];
      Y[i * m + c] = s / L[i * m + i];
    }
  for (int r = 0; r < m; ++r)
    for (int i = 0; i < m; ++i) {
      dd s = Y[r * m + i];
      for (int k = 0; k < i; ++k) s -= L[i * m + k] * S[r * m + k];
      S[r * m + i] = s / L[i * m + i];
    }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      dd avg = (S[i * m + j] + S[j * m + i]) * dd(0.5);
      S[i * m + j] = avg;
      S[j * m + i] = avg;
    }
  std::vector<dd> Q(m * m, dd(0.0));
  for (int i = 0; i < m; ++i) Q[i * m + i] = dd(1.0);
  for (int sweep = 0; sweep < 60; ++sweep) {
    dd off(0.0), tot(0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        dd v = S[i * m + j] * S[i * m + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off.hi <= 1e-62 * tot.hi || off.hi == 0.0) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        dd apq = S[p * m + q];
        // skip rotations that are negligible at double-double precision
        if (std::fabs(apq.hi) <= 1e-34 * std::sqrt(std::fabs(S[p * m + p].hi * S[q * m + q].hi))) continue;
        dd theta = (S[q * m + q] - S[p * m + p]) / (dd(2.0) * apq);
        dd t;
        if (std::fabs(theta.hi) > 1e60) {
          t = dd(0.5) / theta;          // tan of the rotation angle ~ 1 / (2 theta)
        } else {
          t = dd(1.0) / (dd_abs(theta) + dd_sqrt(theta * theta + dd(1.0)));
          if (theta.hi < 0.0) t = -t;
        }
        dd c = dd(1.0) / dd_sqrt(t * t + dd(1.0));
        dd s = t * c;
        for (int k = 0; k < m; ++k) {   // columns p, q
          dd skp = S[k * m + p], skq = S[k * m + q];
          S[k * m + p] = c * skp - s * skq;
          S[k * m + q] = s * skp + c * skq;
        }
        for (int k = 0; k < m; ++k) {   // rows p, q
          dd spk = S[p * m + k], sqk = S[q * m + k];
          S[p * m + k] = c * spk - s * sqk;
          S[q * m + k] = s * spk + c * sqk;
        }
        for (int k = 0; k < m; ++k) {
          dd qkp = Q[k * m + p], qkq = Q[k * m + q];
          Q[k * m + p] = c * qkp - s * qkq;
          Q[k * m + q] = s * qkp + c * qkq;
        }
      }
  }
  // X = L^{-T} Q
  std::vector<dd> Xr(m * m);
  for (int c = 0; c < m; ++c)
    for (int i = m - 1; i >= 0; --i) {
      dd s = Q[i * m + c];
      for (int k = i + 1; k < m; ++k) s -= L[k * m + i] * Xr[k * m + c];
      Xr[i * m + c] = s / L[i * m + i];
    }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return S[a * m + a] < S[b * m + b]; });
  lam->resize(m);
  X->resize(m * m);
  for (int j = 0; j < m; ++j) {
    (*lam)[j] = S[order[j] * m + order[j]];
    for (int i = 0; i < m; ++i) (*X)[i * m + j] = Xr[i * m + order[j]];
  }
  return 0;
}

// -------------------------------------------------------------- axis tables

int interior_eig(int n, std::vector<double>* nu, std::vector<double>* phi) {
  nu->clear();
  phi->clear();
  if (n < 2) return 0;
  std::vector<dd> A, C;
  reference_matrices_dd(n, &A, &C);
  const int n1 = n + 1, m = n - 1;
  std::vector<dd> At(m * m), Ct(m * m), lam, E;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      At[i * m + j] = A[(i + 1) * n1 + (j + 1)];
      Ct[i * m + j] = C[(i + 1) * n1 + (j + 1)];
    }
  if (sym_def_eig(m, At, Ct, &lam, &E)) return -2;
  nu->resize(m);
  phi->resize(m * m);
  for (int l = 0; l < m; ++l) (*nu)[l] = lam[l].to_double();
  for (int i = 0; i < m * m; ++i) (*phi)[i] = E[i].to_double();
  return 0;
}

int precompute_axis(int n, int K, double X, double a, AxisHost* out) {
  if (n < 1 || n > kMaxOrder || K < 2) return -1;
  AxisHost& ax = *out;
  ax.n = n;
  ax.K = K;
  ax.M = n * K - 1;
  ax.X = X;
  ax.a = a;
  ax.h = X / K;
  ax.s = 4.0 / (ax.h * ax.h);
  const int M = ax.M, n1 = n + 1;
  const int Q = n / 2 + 1;          // sine-type sequences (node + even parts)
  const int QC = (n - 1) / 2 + 1;   // cosine-type sequences (node + odd parts)

  std::vector<dd> A, C;
  reference_matrices_dd(n, &A, &C);

  ax.lam.assign(M, 0.0);
  ax.cnorm.assign(M, 0.0);
  ax.mu.assign(M, 0.0);
  ax.tw.assign(2 * K, 0.0);
  ax.rot.assign(2 * K, 0.0);
  const int Q2 = 2 * Q;              // reals per chunk: (sine, cosine) pairs
  ax.fwd.assign((size_t)K * n * Q2, 0.0);
  ax.fwdc.assign((size_t)K * n * Q2, 0.0);
  ax.inv.assign((size_t)K * Q2 * n, 0.0);
  // partition of the reference mass matrix (Section 2): C = [c0 c^T cn; c C~ c^; cn c^T c0]
  std::vector<dd> cvec(std::max(n - 1, 1)), Ct_(std::max((n - 1) * (n - 1), 1));
  for (int i = 0; i + 1 < n; ++i) {
    cvec[i] = C[(i + 1) * n1 + 0];
    for (int j = 0; j + 1 < n; ++j) Ct_[i * (n - 1) + j] = C[(i + 1) * n1 + (j + 1)];
  }
  const dd c0 = C[0], cn = C[n];
  ax.pvec.assign((size_t)K * n * std::max(n - 1, 1), 0.0);
  ax.parity.assign(std::max(n - 1, 0), 0);

  for (int j = 0; j < K; ++j) {
    dd s, c;
    dd_sincospi_frac(2LL * j, K, &s, &c);
    ax.tw[2 * j] = c.to_double();
    ax.tw[2 * j + 1] = -s.to_double();
    dd_sincospi_frac(j, 2LL * K, &s, &c);
    ax.rot[2 * j] = c.to_double();
    ax.rot[2 * j + 1] = -s.to_double();
  }

  // ---- bubble modes: A~ e = lambda C~ e (Section 2), k = 0 of Theorem 1
  if (n >= 2) {
    int m = n - 1;
    std::vector<dd> At(m * m), Ct(m * m), lam0, E;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        At[i * m + j] = A[(i + 1) * n1 + (j + 1)];
        Ct[i * m + j] = C[(i + 1) * n1 + (j + 1)];
      }
    if (sym_def_eig(m, At, Ct, &lam0, &E)) return -2;
    // Section 2, Lemma 1: each e^(l) is even or odd.  Chunk 0 after the FFT
    // holds, for sequence q, slot 2q = S_q(K) (alternating sum) and slot
    // 2q+1 = C_q(0) (plain sum); the bubble maps read/write these slots.
    double* fb = &ax.fwd[0];   // [n-1][2Q]
    double* ib = &ax.inv[0];   // [2Q][n]  (columns l = 0..n-2)
    for (int l = 0; l < m; ++l) {
      double de = 0.0, dodd = 0.0;
      for (int i = 0; i < m; ++i) {
        double ei = E[i * m + l].to_double(), ef = E[(m - 1 - i) * m + l].to_double();
        de += (ei - ef) * (ei - ef);
        dodd += (ei + ef) * (ei + ef);
      }
      int par = de < dodd ? 1 : -1;
      ax.parity[l] = par;
      ax.lam[l] = lam0[l].to_double();
      ax.cnorm[l] = double(K);
      for (int i = 0; i < m; ++i) ax.pvec[(size_t)l * (n - 1) + i] = E[i * m + l].to_double();
      // direct F_n-transform (Theorem 2, item 3): (C w, s_0) = (C~ sum_j (-P)^{j-1} w_{j-1/2}) . e,
      // i.e. the bubble map with C~ e in place of e
      double* fbc = &ax.fwdc[0];
      for (int q = 1; q < Q; ++q) {
        dd ce(0.0);
        for (int i = 0; i < m; ++i) ce += Ct_[(q - 1) * m + i] * E[i * m + l];
        if (par > 0) fbc[l * Q2 + 2 * q] = (ce / dd(double(K))).to_double();
        else if (q < QC) fbc[l * Q2 + 2 * q + 1] = (ce / dd(double(K))).to_double();
      }
      // forward: y_0l = (1/K) sum_m e[m] S_m(K) (even e) or sum_m e[m] C_m(0) (odd e)
      // inverse: a_m(K) = b_e[m], b_m(0) = b_o[m] with b = sum_l w_0l e^(l)
      for (int q = 1; q < Q; ++q) {
        double em = E[(q - 1) * m + l].to_double();
        if (par > 0) {
          fb[l * Q2 + 2 * q] = em / K;
          ib[(2 * q) * n + l] = em;
        } else if (q < QC) {
          fb[l * Q2 + 2 * q + 1] = em / K;
          ib[(2 * q + 1) * n + l] = em;
        }
      }
    }
  }

  // ---- per-frequency modes, Theorem 1 item 3 via the n x n restriction
  // A_theta = (A00 + AJ00) - t AJ00 with t = 1 - theta_k = 2 sin^2(pi k/(2K))
  std::vector<dd> SA(n * n), SC(n * n), AJ(n * n), CJ(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      AJ[i * n + j] = A[i * n1 + (n - j)];
      CJ[i * n + j] = C[i * n1 + (n - j)];
      SA[i * n + j] = A[i * n1 + j] + AJ[i * n + j];
      SC[i * n + j] = C[i * n1 + j] + CJ[i * n + j];
    }
  std::vector<dd> At(n * n), Ct(n * n), lamk, Z;
  for (int k = 1; k < K; ++k) {
    dd sh, chh;
    dd_sincospi_frac(k, 2LL * K, &sh, &chh);      // sin, cos of phi_k = pi k / (2K)
    dd t = dd(2.0) * sh * sh;                      // 1 - cos(pi k / K)
    dd theta = dd(1.0) - t;
    for (int i = 0; i < n * n; ++i) {
      At[i] = SA[i] - t * AJ[i];
      Ct[i] = SC[i] - t * CJ[i];
    }
    if (sym_def_eig(n, At, Ct, &lamk, &Z)) return -2;
    double cphi = chh.to_double(), sphi = sh.to_double();
    double* F = &ax.fwd[(size_t)k * n * Q2];
    double* I = &ax.inv[(size_t)k * Q2 * n];
    for (int l = 0; l < n; ++l) {
      dd z0 = Z[0 * n + l];
      if (z0.hi == 0.0) return -2;
      std::vector<dd> z(n);
      for (int i = 0; i < n; ++i) z[i] = Z[i * n + l] / z0;   // v = 1
      dd nrm(0.0);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) nrm += z[i] * Ct[i * n + j] * z[j];
      nrm = nrm * dd(double(K));
      int sig = n * k - 1 + l;
      ax.lam[sig] = lamk[l].to_double();
      ax.cnorm[sig] = nrm.to_double();
      for (int i = 0; i < n - 1; ++i) ax.pvec[((size_t)k * n + l) * (n - 1) + i] = z[i + 1].to_double();
      // p_e[m] = (p[m] + p[n-m]) / 2, p_o[m] = (p[m] - p[n-m]) / 2 (1-based m;
      // p[m] = z[m]).  Inputs of the forward map at chunk k: slot 2q = 2 S_q(k),
      // slot 2q+1 = 2 C_q(k) (the post-twiddle combination is left doubled):
      //   S_0: cos(phi)/(4N), S_m: cos(phi) p_e[m] / N,
      //   C_0: sin(phi)/(4N), C_m: -sin(phi) p_o[m] / N.
      // Outputs of the inverse map at chunk k: slot 2q = a_q / 2, slot 2q+1 =
      // b_q / 2 (the half of the pre-twiddle combination folded in):
      //   a_0: cos(phi)/2, a_m: cos(phi) p_e[m], b_0: sin(phi)/2, b_m: -sin(phi) p_o[m].
      dd inv_n = dd(1.0) / nrm;
      F[l * Q2 + 0] = (chh * inv_n * dd(0.25)).to_double();
      F[l * Q2 + 1] = (sh * inv_n * dd(0.25)).to_double();
      {
        // direct F_n-transform (Theorem 2, item 3, second formula): the node
        // sum weighted by 2 [c0 + c.p + theta (cn + c.p^)] and p replaced by
        // q = C~ p + c in the interior sums
        double* FC = &ax.fwdc[(size_t)k * n * Q2];
        dd cp(0.0), cpc(0.0);
        std::vector<dd> qz(n + 1, dd(0.0));   // qz[1..n-1] = q (1-based like z)
        for (int i = 0; i + 1 < n; ++i) {
          cp += cvec[i] * z[i + 1];
          cpc += cvec[i] * z[n - 1 - i];
          dd acc = cvec[i];
          for (int j = 0; j + 1 < n; ++j) acc += Ct_[i * (n - 1) + j] * z[j + 1];
          qz[i + 1] = acc;
        }
        const dd gam = dd(2.0) * (c0 + cp + theta * (cn + cpc));
        FC[l * Q2 + 0] = (gam * chh * inv_n * dd(0.25)).to_double();
        FC[l * Q2 + 1] = (gam * sh * inv_n * dd(0.25)).to_double();
        for (int q = 1; q < Q; ++q) {
          FC[l * Q2 + 2 * q] = (chh * ((qz[q] + qz[n - q]) * dd(0.5)) * inv_n).to_double();
          if (q < QC) FC[l * Q2 + 2 * q + 1] = (-(sh * ((qz[q] - qz[n - q]) * dd(0.5)) * inv_n)).to_double();
        }
      }
      I[0 * n + l] = 0.5 * cphi;
      I[1 * n + l] = 0.5 * sphi;
      for (int q = 1; q < Q; ++q) {
        dd pe = (z[q] + z[n - q]) * dd(0.5);
        F[l * Q2 + 2 * q] = (chh * pe * inv_n).to_double();
        I[(2 * q) * n + l] = (chh * pe).to_double();
        if (q < QC) {
          dd po = (z[q] - z[n - q]) * dd(0.5);
          F[l * Q2 + 2 * q + 1] = (-(sh * po * inv_n)).to_double();
          I[(2 * q + 1) * n + l] = (-(sh * po)).to_double();
        }
      }
    }
  }
  for (int i = 0; i < M; ++i) ax.mu[i] = a * ax.s * ax.lam[i];
  fast_tables(&ax);
  return 0;
}

bool fast_schedule(int K, int* V, int* npass, int* radix) {
  if (K < 16 || K > 1024 || (K & (K - 1))) return false;
  const int v = K >= 512 ? 32 : 16;
  int np = 0, rem = K;
  while (rem > 1) {
    const int R = std::min(v, rem);
    radix[np++] = R;
    rem /= R;
  }
  *V = v;
  *npass = np;
  return true;
}

void fast_muk_update(AxisHost* axp) {
  AxisHost& ax = *axp;
  if (!ax.fast_V) return;
  const int n = ax.n, K = ax.K;
  ax.muk.assign((size_t)n * K, 0.0);
  for (int l = 0; l + 1 < n; ++l) ax.muk[(size_t)l * K] = ax.mu[l];
  for (int k = 1; k < K; ++k)
    for (int l = 0; l < n; ++l) ax.muk[(size_t)l * K + k] = ax.mu[n * k - 1 + l];
}

void fast_tables(AxisHost* axp) {
  AxisHost& ax = *axp;
  ax.fast_V = 0;
  int V, np, rad[4];
  if (!fast_schedule(ax.K, &V, &np, rad)) return;
  const int n = ax.n, K = ax.K, Q2 = 2 * (n / 2 + 1);
  ax.fast_V = V;
  ax.fast_npass = np;
  // four-step twiddles between the two passes: tw4[r][i] = exp(-2 pi i r i / K)
  // = tw[r i mod K], r < R0, i < K / R0
  int L = 1;
  for (int s = 0; s < np; ++s) {
    ax.fast_radix[s] = rad[s];
    ax.fast_lprod[s] = L;
    ax.fast_twofs[s] = 0;
    L *= rad[s];
  }
  ax.tw2.assign(2 * (size_t)K, 0.0);
  const int R0 = rad[0], KR = K / R0;
  for (int r = 0; r < R0; ++r)
    for (int i = 0; i < KR; ++i) {
      const int j = (r * i) % K;
      ax.tw2[2 * ((size_t)r * KR + i)] = ax.tw[2 * j];
      ax.tw2[2 * ((size_t)r * KR + i) + 1] = ax.tw[2 * j + 1];
    }
  // G_k[j][l] = the inverse map, frequencies contiguous
  ax.gmap.assign((size_t)Q2 * n * K, 0.0);
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < Q2; ++j)
      for (int l = 0; l < n; ++l) ax.gmap[((size_t)j * n + l) * K + k] = ax.inv[((size_t)k * Q2 + j) * n + l];
  ax.invn.assign((size_t)n * K, 0.0);
  for (int l = 0; l + 1 < n; ++l) ax.invn[(size_t)l * K] = 1.0 / K;
  for (int k = 1; k < K; ++k)
    for (int l = 0; l < n; ++l) ax.invn[(size_t)l * K + k] = 1.0 / ax.cnorm[n * k - 1 + l];
  fast_muk_update(&ax);
}

}  // namespace femfft
