// Host FP64 linear algebra for the projected problem of eq. (proj).
//
// The paper solves T_k W_k = W_k Lambda_k on the CPU with a banded symmetric
// eigensolver (Section 3.2.2): T_k is block tridiagonal, i.e. symmetric with
// semi-bandwidth r. Here:
//   * eigenvalues: orthogonal band-to-tridiagonal reduction by Givens
//     rotations with bulge chasing (O(K^2 r)), then implicit QL with the
//     Wilkinson shift on the tridiagonal (O(K^2));
//   * eigenvectors, only for the Ritz pairs the convergence test inspects:
//     inverse iteration on the band matrix itself with a partial-pivoting band
//     LU (O(K r^2) per solve), orthogonalizing the vectors of close
//     eigenvalues against each other.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "flz_internal.h"

namespace flz {

namespace {

inline void rotate_rows(double* T, int K, int p, int q, double c, double s, int j0, int j1) {
  double* rp = T + (size_t)p * K;
  double* rq = T + (size_t)q * K;
  for (int j = j0; j <= j1; ++j) {
    const double x = rp[j], y = rq[j];
    rp[j] = c * x + s * y;
    rq[j] = -s * x + c * y;
  }
}

inline void rotate_cols(double* T, int K, int p, int q, double c, double s, int i0, int i1) {
  for (int i = i0; i <= i1; ++i) {
    double* row = T + (size_t)i * K;
    const double x = row[p], y = row[q];
    row[p] = c * x + s * y;
    row[q] = -s * x + c * y;
  }
}

// Zero T[k][j] (and T[j][k]) by a rotation in the plane (k-1, k) applied as a
// similarity transform; entries outside [k-1-w, k+w] of rows/cols k-1, k are 0.
inline void annihilate(double* T, int K, int k, int j, int w) {
  const double x = T[(size_t)(k - 1) * K + j];
  const double y = T[(size_t)k * K + j];
  if (y == 0.0) return;
  const double r = std::hypot(x, y);
  const double c = x / r, s = y / r;
  const int lo = std::max(0, k - 1 - w), hi = std::min(K - 1, k + w);
  rotate_rows(T, K, k - 1, k, c, s, lo, hi);
  rotate_cols(T, K, k - 1, k, c, s, lo, hi);
  T[(size_t)k * K + j] = 0.0;
  T[(size_t)j * K + k] = 0.0;
}

}  // namespace

void tridiagonal_eigenvalues(std::vector<double>& d, std::vector<double>& e) {
  // Implicit QL with the Wilkinson shift. e[i] couples i and i+1; e.size() >= d.size().
  const int K = (int)d.size();
  e.resize(std::max<size_t>(e.size(), (size_t)K));
  if (K > 0) e[K - 1] = 0.0;
  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < K; ++l) {
    for (int iter = 0; iter < 200; ++iter) {
      int m = l;
      for (; m < K - 1; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      // Shift: eigenvalue of the leading 2x2 of the unreduced block closest to d[l].
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool deflated = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i];
        const double bb = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * bb;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - bb;
      }
      if (deflated) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  std::sort(d.begin(), d.end());
}

void band_eigenvalues(const std::vector<double>& Tin, int K, int b, std::vector<double>& theta) {
  std::vector<double> T(Tin);
  const int w = 2 * b + 2;
  if (b > 1) {
    for (int j = 0; j + 2 < K; ++j) {
      for (int k = std::min(j + b, K - 1); k >= j + 2; --k) {
        annihilate(T.data(), K, k, j, w);
        // Chase the bulge created at (k + b, k - 1) down the band.
        int col = k - 1, q = k + b;
        while (q < K) {
          annihilate(T.data(), K, q, col, w);
          col = q - 1;
          q += b;
        }
      }
    }
  }
  std::vector<double> d(K), e(K, 0.0);
  for (int i = 0; i < K; ++i) d[i] = T[(size_t)i * K + i];
  for (int i = 0; i + 1 < K; ++i) e[i] = T[(size_t)(i + 1) * K + i];
  tridiagonal_eigenvalues(d, e);
  theta = d;
}

namespace {

struct BandLU {
  int K = 0, b = 0, W = 0;
  std::vector<double> U;  // U(i, j) at U[i*W + (j - i + b)], j - i in [-b, 2b]
  std::vector<double> L;  // multipliers, L[k*b + (i - k - 1)]
  std::vector<int> piv;
  double& u(int i, int j) { return U[(size_t)i * W + (j - i + b)]; }
};

void band_lu(const std::vector<double>& T, int K, int b, double shift, double tiny, BandLU& f) {
  f.K = K;
  f.b = b;
  f.W = 3 * b + 1;
  f.U.assign((size_t)K * f.W, 0.0);
  f.L.assign((size_t)K * std::max(b, 1), 0.0);
  f.piv.assign(K, 0);
  for (int i = 0; i < K; ++i)
    for (int j = std::max(0, i - b); j <= std::min(K - 1, i + b); ++j)
      f.u(i, j) = T[(size_t)i * K + j] - (i == j ? shift : 0.0);
  for (int k = 0; k < K; ++k) {
    const int last = std::min(K - 1, k + b);
    int p = k;
    double best = std::fabs(f.u(k, k));
    for (int i = k + 1; i <= last; ++i)
      if (std::fabs(f.u(i, k)) > best) {
        best = std::fabs(f.u(i, k));
        p = i;
      }
    f.piv[k] = p;
    const int jend = std::min(K - 1, k + 2 * b);
    if (p != k)
      for (int j = k; j <= jend; ++j) std::swap(f.u(k, j), f.u(p, j));
    if (std::fabs(f.u(k, k)) < tiny) f.u(k, k) = std::copysign(tiny, f.u(k, k) == 0.0 ? 1.0 : f.u(k, k));
    const double piv = f.u(k, k);
    for (int i = k + 1; i <= last; ++i) {
      const double l = f.u(i, k) / piv;
      f.L[(size_t)k * b + (i - k - 1)] = l;
      if (l != 0.0)
        for (int j = k + 1; j <= jend; ++j) f.u(i, j) -= l * f.u(k, j);
      f.u(i, k) = 0.0;
    }
  }
}

void band_solve(BandLU& f, double* x) {
  const int K = f.K, b = f.b;
  for (int k = 0; k < K; ++k) {
    if (f.piv[k] != k) std::swap(x[k], x[f.piv[k]]);
    const int last = std::min(K - 1, k + b);
    for (int i = k + 1; i <= last; ++i) x[i] -= f.L[(size_t)k * b + (i - k - 1)] * x[k];
  }
  for (int k = K - 1; k >= 0; --k) {
    double s = x[k];
    const int jend = std::min(K - 1, k + 2 * b);
    for (int j = k + 1; j <= jend; ++j) s -= f.u(k, j) * x[j];
    x[k] = s / f.u(k, k);
  }
}

inline uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

void band_eigenvectors(const std::vector<double>& T, int K, int b, const std::vector<double>& theta,
                       const std::vector<int>& idx, std::vector<double>& Y, uint64_t seed) {
  const int cnt = (int)idx.size();
  Y.assign((size_t)K * cnt, 0.0);
  double tnorm = 0.0;
  for (int i = 0; i < K; ++i) {
    double s = 0.0;
    for (int j = std::max(0, i - b); j <= std::min(K - 1, i + b); ++j) s += std::fabs(T[(size_t)i * K + j]);
    tnorm = std::max(tnorm, s);
  }
  if (tnorm == 0.0) tnorm = 1.0;
  const double eps = 2.220446049250313e-16;
  const double tiny = eps * tnorm;
  const double close = 1e-3 * tnorm;
  // Process in order of the requested eigenvalues; vectors of eigenvalues
  // within `close` of each other are orthogonalized against earlier ones.
  std::vector<int> order(cnt);
  for (int t = 0; t < cnt; ++t) order[t] = t;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return theta[idx[x]] < theta[idx[y]]; });
  BandLU f;
  std::vector<double> x(K);
  for (int oi = 0; oi < cnt; ++oi) {
    const int t = order[oi];
    const double lam = theta[idx[t]];
    band_lu(T, K, b, lam, tiny, f);
    uint64_t st = mix64(seed ^ (uint64_t)(idx[t] + 1) * 0x2545F4914F6CDD1Dull);
    for (int i = 0; i < K; ++i) {
      st = mix64(st);
      x[i] = ((double)(st >> 11) * (1.0 / 9007199254740992.0)) - 0.5;
    }
    for (int it = 0; it < 4; ++it) {
      band_solve(f, x.data());
      // orthogonalize against already computed vectors of close eigenvalues
      for (int pj = oi - 1; pj >= 0; --pj) {
        const int tp = order[pj];
        if (lam - theta[idx[tp]] > close) break;
        const double* yp = &Y[(size_t)tp * K];
        double dot = 0.0;
        for (int i = 0; i < K; ++i) dot += yp[i] * x[i];
        for (int i = 0; i < K; ++i) x[i] -= dot * yp[i];
      }
      double nrm = 0.0;
      for (int i = 0; i < K; ++i) nrm += x[i] * x[i];
      nrm = std::sqrt(nrm);
      if (nrm == 0.0) nrm = 1.0;
      for (int i = 0; i < K; ++i) x[i] /= nrm;
    }
    std::memcpy(&Y[(size_t)t * K], x.data(), sizeof(double) * K);
  }
}

bool cholesky_upper(const double* G, int s, double* R) {
  for (int i = 0; i < s * s; ++i) R[i] = 0.0;
  for (int i = 0; i < s; ++i) {
    double dsum = G[i * s + i];
    for (int k = 0; k < i; ++k) dsum -= R[k * s + i] * R[k * s + i];
    if (!(dsum > 0.0)) return false;
    const double rii = std::sqrt(dsum);
    R[i * s + i] = rii;
    for (int j = i + 1; j < s; ++j) {
      double v = G[i * s + j];
      for (int k = 0; k < i; ++k) v -= R[k * s + i] * R[k * s + j];
      R[i * s + j] = v / rii;
    }
  }
  return true;
}

void upper_inverse(const double* R, int s, double* Rinv) {
  for (int i = 0; i < s * s; ++i) Rinv[i] = 0.0;
  for (int j = 0; j < s; ++j) {
    Rinv[j * s + j] = 1.0 / R[j * s + j];
    for (int i = j - 1; i >= 0; --i) {
      double v = 0.0;
      for (int k = i + 1; k <= j; ++k) v += R[i * s + k] * Rinv[k * s + j];
      Rinv[i * s + j] = -v / R[i * s + i];
    }
  }
}

}  // namespace flz
