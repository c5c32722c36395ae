// Host-side layout choice of the register-radix pencil passes
// (pencil_fast.cuh): a model of the shared-memory bank accesses of one tile
// (8-byte complex words, served per half-warp: a request costs, per half,
// the largest number of distinct words that fall in one of the 16 bank
// pairs) over the two FFT directions and the map phase, minimised over the
// sequence order, the pencil pitch and the swizzle of the FFT's intermediate
// buffers.  Cached per shape.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.h"

namespace femfft {
namespace {

int makhoul(int r, int K) { return r < K / 2 ? 2 * r : 2 * (K - 1 - r) + 1; }
int swz(int e, int sh) { return sh ? (e ^ ((e >> sh) & ((1 << (sh < 4 ? sh : 4)) - 1))) : e; }

// wavefronts of one warp-wide request (-1: inactive lane)
int wavefronts(const long long* a) {
  int total = 0;
  for (int h = 0; h < 2; ++h) {
    int worst = 0;
    bool any = false;
    for (int i = 0; i < 16; ++i) {
      const long long x = a[16 * h + i];
      if (x < 0) continue;
      any = true;
      int distinct = 0;
      for (int j = 0; j < 16; ++j) {
        const long long y = a[16 * h + j];
        if (y < 0 || (y & 15) != (x & 15)) continue;
        bool seen = false;
        for (int m = 0; m < j; ++m)
          if (a[16 * h + m] == y) seen = true;
        if (!seen) ++distinct;
      }
      worst = std::max(worst, distinct);
    }
    total += any ? worst : 0;
  }
  return total;
}

struct Cost {
  long long waves = 0, ideal = 0;
  void add(const long long* a) {
    const int w = wavefronts(a);
    if (!w) return;
    waves += w;
    for (int h = 0; h < 2; ++h)
      for (int i = 0; i < 16; ++i)
        if (a[16 * h + i] >= 0) {
          ++ideal;
          break;
        }
  }
};

// the accesses of fast_fft (both Makhoul directions)
void model_fft(int K, int Q, int Qp, int W, int V, int npass, const int* radix, int nthreads, int order, int pitch,
               const int* sh, bool perm_in, bool perm_out, Cost* c) {
  const int Tn = K / V, nseq = W * Q, spr = nthreads / Tn;
  long long a[32];
  for (int s0 = 0; s0 < nseq; s0 += spr) {
    for (int w = 0; w < nthreads / 32; ++w) {
      int L = 1;
      for (int ps = 0; ps < npass; ++ps) {
        const int R = radix[ps], G = V / R;
        for (int wr = 0; wr < 2; ++wr)
          for (int g = 0; g < G; ++g)
            for (int r = 0; r < R; ++r) {
              for (int ln = 0; ln < 32; ++ln) {
                const int t = w * 32 + ln, sl = t / Tn, tau = t - sl * Tn, seq = s0 + sl;
                if (sl >= spr || seq >= nseq) {
                  a[ln] = -1;
                  continue;
                }
                int pen, q;
                if (order == 0) {
                  pen = seq / Q;
                  q = seq - pen * Q;
                } else {
                  q = seq / W;
                  pen = seq - q * W;
                }
                const int i = tau + g * Tn;
                int pos;
                if (!wr) {
                  const int e = i + r * (K / R);
                  pos = ps == 0 ? (perm_in ? makhoul(e, K) : e) : swz(e, sh[ps - 1]);
                } else {
                  const int k = i % L, e = (i - k) * R + k + r * L;
                  pos = ps == npass - 1 ? (perm_out ? makhoul(e, K) : e) : swz(e, sh[ps]);
                }
                a[ln] = (long long)pen * pitch + q + (long long)pos * Qp;
              }
              c->add(a);
            }
        L *= R;
      }
    }
  }
}

// the chunk reads and writes of fast_maps: task = (pair, pencil), pencil fastest
void model_maps(int K, int Q, int Qp, int W, int nthreads, int pitch, Cost* c) {
  const int ntask = W * (K / 2);
  long long a[32];
  for (int r0 = 0; r0 < ntask; r0 += nthreads)
    for (int w = 0; w < nthreads / 32; ++w)
      for (int which = 0; which < 2; ++which)
        for (int q = 0; q < Q; ++q) {
          for (int ln = 0; ln < 32; ++ln) {
            const int task = r0 + w * 32 + ln;
            if (task >= ntask) {
              a[ln] = -1;
              continue;
            }
            const int tau = task / W, p = task - tau * W;
            const int k = which == 0 ? tau : (tau ? K - tau : K / 2);
            a[ln] = (long long)p * pitch + (long long)k * Qp + q;
          }
          c->add(a);
          c->add(a);   // read and write
        }
}

}  // namespace

void fast_layout(int K, int Q, int Qp, int W, int V, int npass, const int* radix, int nthreads, int* order, int* pitch,
                 int* swzo) {
  typedef std::tuple<int, int, int, int, int, int> Key;
  static std::mutex mu;
  static std::map<Key, std::vector<int>> cache;
  const Key key(K, Q, Qp, W, V, nthreads);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *order = it->second[0];
      *pitch = it->second[1];
      for (int s = 0; s < kFastMaxPass; ++s) swzo[s] = it->second[2 + s];
      return;
    }
  }
  const int cand[5] = {0, 2, 3, 4, 5};
  const int nsw = npass > 1 ? 5 : 1;
  double best = 1e30;
  std::vector<int> pick(2 + kFastMaxPass, 0);
  for (int od = 0; od < 2; ++od) {
    if (od == 1 && W == 1) continue;
    for (int d = 0; d < 16; ++d) {
      const int pt = K * Qp + d;
      Cost cm;
      model_maps(K, Q, Qp, W, nthreads, pt, &cm);
      for (int si = 0; si < nsw; ++si) {
        int sh[kFastMaxPass] = {0, 0, 0, 0};
        for (int s = 0; s + 1 < npass; ++s) sh[s] = cand[si];
        Cost c = cm;
        model_fft(K, Q, Qp, W, V, npass, radix, nthreads, od, pt, sh, true, false, &c);
        model_fft(K, Q, Qp, W, V, npass, radix, nthreads, od, pt, sh, false, true, &c);
        const double cost = double(c.waves) / double(std::max<long long>(1, c.ideal));
        if (cost < best - 1e-9) {
          best = cost;
          pick[0] = od;
          pick[1] = pt;
          for (int s = 0; s < kFastMaxPass; ++s) pick[2 + s] = sh[s];
        }
      }
    }
  }
  *order = pick[0];
  *pitch = pick[1];
  for (int s = 0; s < kFastMaxPass; ++s) swzo[s] = pick[2 + s];
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = pick;
}

}  // namespace femfft
