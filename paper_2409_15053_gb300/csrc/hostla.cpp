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

}  // namespace

// sqrt(x^2 + y^2); the projected matrices have entries of order ||p(A)|| or
// ||A||, far from the overflow range that std::hypot guards against (and
// std::hypot costs several times more, in the innermost QL loop).
static inline double pyth(double x, double y) { return std::sqrt(x * x + y * y); }

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
      double r = pyth(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool deflated = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i];
        const double bb = c * e[i];
        r = pyth(f, g);
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
  // Compact lower-band storage with one extra diagonal for the bulge:
  // A[i*W + d] = T[i][i-d], d in [0, b+1].
  const int W = b + 2;
  std::vector<double> A((size_t)K * W, 0.0);
  for (int i = 0; i < K; ++i)
    for (int d = 0; d <= std::min(b, i); ++d) A[(size_t)i * W + d] = Tin[(size_t)i * K + (i - d)];
  auto at = [&](int i, int d) -> double& { return A[(size_t)i * W + d]; };
  // Similarity rotation in the plane (q, q+1) chosen to zero T[q+1][jj]; the
  // rows and columns it touches hold nonzeros only in [jj, q+1+b].
  auto rotate = [&](int q, int jj) {
    const int p = q + 1;
    const double x = at(q, q - jj), y = at(p, p - jj);
    if (y == 0.0) return;
    const double r = pyth(x, y), c = x / r, s = y / r;
    for (int xc = jj + 1; xc <= q - 1; ++xc) {
      const double u = at(q, q - xc), v = at(p, p - xc);
      at(q, q - xc) = c * u + s * v;
      at(p, p - xc) = -s * u + c * v;
    }
    at(q, q - jj) = r;
    at(p, p - jj) = 0.0;
    const double a = at(q, 0), bb = at(p, 1), d = at(p, 0);
    at(q, 0) = c * c * a + 2.0 * c * s * bb + s * s * d;
    at(p, 0) = s * s * a - 2.0 * c * s * bb + c * c * d;
    at(p, 1) = -c * s * a + (c * c - s * s) * bb + c * s * d;
    const int xe = std::min(K - 1, p + b);
    for (int xr = p + 1; xr <= xe; ++xr) {
      const double u = at(xr, xr - q), v = at(xr, xr - p);
      at(xr, xr - q) = c * u + s * v;
      at(xr, xr - p) = -s * u + c * v;
    }
  };
  if (b > 1) {
    for (int j = 0; j + 2 < K; ++j) {
      for (int k = std::min(j + b, K - 1); k >= j + 2; --k) {
        rotate(k - 1, j);
        // chase the bulge at (k + b, k - 1) down the band
        int col = k - 1, q = k + b - 1;
        while (q + 1 < K) {
          rotate(q, col);
          col = q;
          q += b;
        }
      }
    }
  }
  std::vector<double> dg(K), e(K, 0.0);
  for (int i = 0; i < K; ++i) dg[i] = at(i, 0);
  for (int i = 0; i + 1 < K; ++i) e[i] = at(i + 1, 1);
  tridiagonal_eigenvalues(dg, e);
  theta = dg;
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
                       const std::vector<int>& idx, std::vector<double>& Y, uint64_t seed,
                       const std::vector<double>* prevY, const std::vector<int>* prevIdx) {
  const int nprev = prevIdx ? (int)prevIdx->size() : 0;
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
  // Vectors are computed in the order of `idx`, each orthogonalized against
  // every earlier one -- of this call, and the given vectors of earlier calls
  // (prevY, columns for prevIdx) -- whose eigenvalue lies within `close`: the
  // copies of a multiple or tightly clustered eigenvalue stay orthogonal when
  // they are requested in different calls.
  BandLU f;
  std::vector<double> x(K);
  for (int t = 0; t < cnt; ++t) {
    const double lam = theta[idx[t]];
    band_lu(T, K, b, lam, tiny, f);
    uint64_t st = mix64(seed ^ (uint64_t)(idx[t] + 1) * 0x2545F4914F6CDD1Dull);
    for (int i = 0; i < K; ++i) {
      st = mix64(st);
      x[i] = ((double)(st >> 11) * (1.0 / 9007199254740992.0)) - 0.5;
    }
    for (int it = 0; it < 4; ++it) {
      band_solve(f, x.data());
      for (int tp = 0; tp < nprev; ++tp) {
        if (std::fabs(lam - theta[(*prevIdx)[tp]]) > close) continue;
        const double* yp = &(*prevY)[(size_t)tp * K];
        double dot = 0.0;
        for (int i = 0; i < K; ++i) dot += yp[i] * x[i];
        for (int i = 0; i < K; ++i) x[i] -= dot * yp[i];
      }
      for (int tp = 0; tp < t; ++tp) {
        if (std::fabs(lam - theta[idx[tp]]) > close) continue;
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

namespace flz {

// Dense symmetric eigen-decomposition (Golub & Van Loan: Householder
// tridiagonalization with the orthogonal factor accumulated, then implicit QL
// with the Wilkinson shift, every rotation applied to the accumulated basis).
// A: n x n row-major symmetric (destroyed). w: eigenvalues ascending;
// Z: n x n row-major with column k the unit eigenvector of w[k].
void dense_sym_eig(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& Z) {
  Z.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), p(n), q(n);
  for (int k = 0; k + 2 < n; ++k) {
    // reflector H = I - beta v v^T mapping A[k+1:, k] to a multiple of e_1
    double sigma = 0.0;
    for (int i = k + 2; i < n; ++i) sigma += A[(size_t)i * n + k] * A[(size_t)i * n + k];
    const double x0 = A[(size_t)(k + 1) * n + k];
    if (sigma == 0.0) continue;
    const double mu = std::sqrt(x0 * x0 + sigma);
    const double v0 = x0 <= 0.0 ? x0 - mu : -sigma / (x0 + mu);
    const double beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
    v[k + 1] = 1.0;
    for (int i = k + 2; i < n; ++i) v[i] = A[(size_t)i * n + k] / v0;
    // p = beta * A22 v ; w = p - (beta/2)(p^T v) v ; A22 -= v w^T + w v^T
    for (int i = k + 1; i < n; ++i) {
      double s = 0.0;
      const double* row = &A[(size_t)i * n];
      for (int j = k + 1; j < n; ++j) s += row[j] * v[j];
      p[i] = beta * s;
    }
    double pv = 0.0;
    for (int i = k + 1; i < n; ++i) pv += p[i] * v[i];
    for (int i = k + 1; i < n; ++i) q[i] = p[i] - 0.5 * beta * pv * v[i];
    for (int i = k + 1; i < n; ++i) {
      double* row = &A[(size_t)i * n];
      for (int j = k + 1; j < n; ++j) row[j] -= v[i] * q[j] + q[i] * v[j];
    }
    const double newsub = mu;  // H x = ||x|| e_1 for either form of v_1
    A[(size_t)(k + 1) * n + k] = newsub;
    A[(size_t)k * n + k + 1] = newsub;
    for (int i = k + 2; i < n; ++i) A[(size_t)i * n + k] = A[(size_t)k * n + i] = 0.0;
    // Z <- Z H (columns k+1..n-1)
    for (int i = 0; i < n; ++i) {
      double* zr = &Z[(size_t)i * n];
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += zr[j] * v[j];
      s *= beta;
      for (int j = k + 1; j < n; ++j) zr[j] -= s * v[j];
    }
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = A[(size_t)(i + 1) * n + i];
  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0; iter < 200; ++iter) {
      int m = l;
      for (; m < n - 1; ++m)
        if (std::fabs(e[m]) <= eps * (std::fabs(d[m]) + std::fabs(d[m + 1]))) break;
      if (m == l) break;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = pyth(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
      double s = 1.0, c = 1.0, pp = 0.0;
      bool deflated = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i], bb = c * e[i];
        r = pyth(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= pp;
          e[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * bb;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - bb;
        for (int k2 = 0; k2 < n; ++k2) {  // rotate columns i, i+1 of Z
          double* zr = &Z[(size_t)k2 * n];
          const double zf = zr[i + 1];
          zr[i + 1] = s * zr[i] + c * zf;
          zr[i] = c * zr[i] - s * zf;
        }
      }
      if (deflated) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  // sort ascending with the columns of Z
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
  w.resize(n);
  std::vector<double> Zs((size_t)n * n);
  for (int k = 0; k < n; ++k) {
    w[k] = d[ord[k]];
    for (int i = 0; i < n; ++i) Zs[(size_t)i * n + k] = Z[(size_t)i * n + ord[k]];
  }
  Z.swap(Zs);
}

}  // namespace flz
