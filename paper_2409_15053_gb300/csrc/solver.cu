// The filtered Lanczos procedure (Sections 2.2, 2.3, 3.2.2) on one GPU.
//
//   bounds      block Lanczos on A (Section 2.2 after eq. transf): extreme Ritz
//               values padded by their residual bounds, clamped to Gershgorin
//   map/filter  eq. (transf), eq. (optimaldegree), closed-form coefficients
//   loop        W = p(A) Q_j (filter.cu); full reorthogonalization of W against
//               the whole basis by classical Gram-Schmidt applied twice;
//               D_j = Q_j^T p(A) Q_j from the two projections; block QR of W by
//               CholeskyQR2 (shifted CholeskyQR3 when W is ill conditioned)
//               giving Q_{j+1} and the upper-triangular S_j (eq. lanczos)
//   check       every `check_every` blocks: T_k (eq. lanczos) on the host,
//               its eigenvalues (eq. proj) by band reduction + QL, Ritz pairs
//               ranked by the p(A) Ritz value; for the leading ones, Ritz
//               vectors Q_k y on the GPU, Rayleigh quotients (eq. rayleigh)
//               and true residuals ||Ax - lambda x|| / ||A||. Converged when every
//               pair with lambda in [alpha, beta] and the `guard` nearest
//               outside have residual <= tol and the count in [alpha, beta] is
//               unchanged since the previous check (Section 3.2.2).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <type_traits>

#include "flz_internal.h"

namespace flz {

namespace {

using Clock = std::chrono::steady_clock;
inline double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

// Host copies of the small per-step matrices of eq. (lanczos).
struct Projected {
  int r = 0;
  std::vector<std::vector<double>> D, S;  // r x r row-major each
  // T_k from D_0..D_{k-1}, S_0..S_{k-2}, symmetrized; dense K x K row-major.
  std::vector<double> assemble(int k) const {
    const int K = k * r;
    std::vector<double> T((size_t)K * K, 0.0);
    for (int b = 0; b < k; ++b) {
      for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j)
          T[(size_t)(b * r + i) * K + b * r + j] = 0.5 * (D[b][i * r + j] + D[b][j * r + i]);
      if (b + 1 < k)
        for (int i = 0; i < r; ++i)
          for (int j = 0; j < r; ++j) {
            const double v = S[b][i * r + j];
            T[(size_t)((b + 1) * r + i) * K + b * r + j] = v;
            T[(size_t)(b * r + j) * K + (b + 1) * r + i] = v;
          }
    }
    return T;
  }
};

// One block Lanczos engine over a basis stored as T: FP64, or double-FP32
// pairs (dev::dfloat) whose inner products and updates run on the FP32 pipes.
// The small matrices (C, D_j, S_j, R^{-1}) are FP64 throughout.
template <class T>
struct Engine {
  flz_matrix* A;
  int64_t n;
  int r;
  cudaStream_t st;
  T* Q;          // basis, nb_cap blocks
  int nb_cap;
  T* W;          // n x r
  double* C;     // nb_cap*r x r
  double* C2;
  double* part;  // basis_dot scratch
  double* small; // device r x r scratch (R^{-1})
  double ms_orth = 0.0, ms_op = 0.0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  TcBasis* tcb = nullptr;  // digit copy of an FP64 basis: reorthogonalization on the tensor cores
  bool fx = false;         // the filter runs in fixed point: check its overflow flag after each step
  // FP64 basis: the block QR runs on the device (scratch qrs) and a step's
  // D_j and S_j reach the host through `pinned` (3 r x r words) at its one
  // synchronization
  double* pinned = nullptr;
  double* qrs = nullptr;

  T* block(int b) const { return Q + (size_t)b * n * r; }

  // Block b of the basis is final: round it to the digit grid and record its digits.
  void seal(int b) {
    if constexpr (std::is_same<T, double>::value)
      if (tcb) tcb->append(block(b), r, b * r, st);
  }

  void gram(const T* X, std::vector<double>& G) {
    basis_dot(X, 1, n, r, X, r, r, C2, part, st);
    G.resize((size_t)r * r);
    FLZ_CUDA(cudaMemcpyAsync(G.data(), C2, sizeof(double) * r * r, cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
  }

  // Out = X R^{-1} (in place allowed).
  void right_solve(const T* X, const std::vector<double>& Rinv, T* Out) {
    FLZ_CUDA(cudaMemcpyAsync(small, Rinv.data(), sizeof(double) * r * r, cudaMemcpyHostToDevice, st));
    basis_update(X, 1, n, r, small, r, 1.0, 0.0, Out, r, st);
  }

  // Block QR of the n x r block X into Out (CholeskyQR2, shifted CholeskyQR3
  // when the first Cholesky fails); returns S (upper triangular, row-major).
  std::vector<double> block_qr(const T* X, T* Out) {
    std::vector<double> G, R((size_t)r * r), Rinv((size_t)r * r), S((size_t)r * r, 0.0), tmp((size_t)r * r);
    for (int i = 0; i < r; ++i) S[i * r + i] = 1.0;
    gram(X, G);
    const T* src = X;
    int passes = 2;
    if (!cholesky_upper(G.data(), r, R.data())) {
      // shifted Cholesky keeps the factorization defined for ill-conditioned X
      double gnorm = 0.0;
      for (int i = 0; i < r; ++i) gnorm = std::max(gnorm, G[i * r + i]);
      gnorm = std::max(gnorm * r, 1e-300);
      const double shift = 11.0 * ((double)n * r + (double)r * (r + 1)) * 1.1102230246251565e-16 * gnorm;
      for (int i = 0; i < r; ++i) G[i * r + i] += shift;
      if (!cholesky_upper(G.data(), r, R.data())) {
        for (int i = 0; i < r * r; ++i) R[i] = 0.0;
        for (int i = 0; i < r; ++i) R[i * r + i] = std::sqrt(std::max(G[i * r + i], 1e-300));
      }
      passes = 3;
    }
    for (int pass = 0; pass < passes; ++pass) {
      if (pass > 0) {
        gram(Out, G);
        if (!cholesky_upper(G.data(), r, R.data())) {
          for (int i = 0; i < r * r; ++i) R[i] = 0.0;
          for (int i = 0; i < r; ++i) R[i * r + i] = std::sqrt(std::max(G[i * r + i], 1e-300));
        }
      }
      upper_inverse(R.data(), r, Rinv.data());
      right_solve(src, Rinv, Out);
      src = Out;
      // S <- R S
      for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
          double v = 0.0;
          for (int k = 0; k < r; ++k) v += R[i * r + k] * S[k * r + j];
          tmp[i * r + j] = v;
        }
      S = tmp;
    }
    return S;
  }

  // Block QR of X into Out on the device (qr_device); S is left at qrs + 256.
  void block_qr_device(const double* X, double* Out) { qr_device(X, Out, n, r, qrs, st); }

  // Classical Gram-Schmidt twice of X against blocks 0..nb-1; returns the
  // total projection coefficients of the last block (r x r, row-major) in Dlast.
  void cgs2(T* X, int nb, std::vector<double>* Dlast) {
    bool done = false;
    if constexpr (std::is_same<T, double>::value)
      if (tcb) {
        tcb->cgs2(nb * r, X, r, C, C2, st);
        done = true;
      }
    if (!done) {
      basis_dot(Q, nb, n, r, X, r, r, C, part, st);
      basis_update(Q, nb, n, r, C, r, -1.0, 1.0, X, r, st);
      basis_dot(Q, nb, n, r, X, r, r, C2, part, st);
      basis_update(Q, nb, n, r, C2, r, -1.0, 1.0, X, r, st);
    }
    if (Dlast) {
      std::vector<double> d1((size_t)r * r), d2((size_t)r * r);
      const size_t off = (size_t)(nb - 1) * r * r;
      FLZ_CUDA(cudaMemcpyAsync(d1.data(), C + off, sizeof(double) * r * r, cudaMemcpyDeviceToHost, st));
      FLZ_CUDA(cudaMemcpyAsync(d2.data(), C2 + off, sizeof(double) * r * r, cudaMemcpyDeviceToHost, st));
      FLZ_CUDA(cudaStreamSynchronize(st));
      Dlast->resize((size_t)r * r);
      for (int i = 0; i < r * r; ++i) (*Dlast)[i] = d1[i] + d2[i];
    }
  }

  // One block Lanczos step j: W = op(Q_j), reorthogonalize, QR into Q_{j+1}.
  // Returns false if the new block could not be formed (no slot).
  // With the device QR a step splits in two halves: step_issue queues all of
  // its GPU work (no host wait); step_finish waits for it, takes D_j and S_j
  // and handles a breakdown. The solver issues the next step before a
  // convergence check's host work, so the two overlap.
  bool issued = false;
  bool can_split() const {
    if constexpr (std::is_same<T, double>::value) return pinned != nullptr;
    return false;
  }
  void step_issue(int j, const std::function<void(const T*, T*)>& op) {
    if (!ev[0])
      for (auto& x : ev) FLZ_CUDA(cudaEventCreate(&x));
    FLZ_CUDA(cudaEventRecord(ev[0], st));
    op(block(j), W);
    FLZ_CUDA(cudaEventRecord(ev[1], st));
    if constexpr (std::is_same<T, double>::value) {
      T* next = (j + 1 < nb_cap) ? block(j + 1) : nullptr;
      cgs2(W, j + 1, nullptr);
      block_qr_device(W, next ? next : W);
      if (next) seal(j + 1);
      const size_t rr = (size_t)r * r, off = (size_t)j * rr;
      FLZ_CUDA(cudaMemcpyAsync(pinned, C + off, sizeof(double) * rr, cudaMemcpyDeviceToHost, st));
      FLZ_CUDA(cudaMemcpyAsync(pinned + rr, C2 + off, sizeof(double) * rr, cudaMemcpyDeviceToHost, st));
      FLZ_CUDA(cudaMemcpyAsync(pinned + 2 * rr, qrs + 256, sizeof(double) * rr, cudaMemcpyDeviceToHost, st));
    }
    FLZ_CUDA(cudaEventRecord(ev[2], st));
    issued = true;
  }
  // keep = false: the step's results are not wanted (the solve stopped at the
  // check it overlapped); it is only waited for, and its time counts in the
  // solve's total but not in the filter and orthogonalization phases (which
  // stay the time of the `iters` steps the results come from)
  void step_finish(int j, Projected& P, double op_norm, bool keep = true) {
    FLZ_CUDA(cudaEventSynchronize(ev[2]));
    issued = false;
    if constexpr (std::is_same<T, double>::value) {
      if (keep) {
        T* next = (j + 1 < nb_cap) ? block(j + 1) : nullptr;
        const size_t rr = (size_t)r * r;
        std::vector<double> D(rr), S(pinned + 2 * rr, pinned + 3 * rr);
        for (size_t i = 0; i < rr; ++i) D[i] = pinned[i] + pinned[rr + i];
        P.D.push_back(D);
        // breakdown: the new block is (nearly) dependent on the basis; its
        // directions are rounding noise and must be made orthogonal to the basis.
        double smin = 1e300;
        for (int i = 0; i < r; ++i) smin = std::min(smin, std::fabs(S[i * r + i]));
        if (next && smin < 1e-12 * std::max(op_norm, 1e-300)) {
          cgs2(next, j + 1, nullptr);
          block_qr_device(next, next);
          seal(j + 1);
          FLZ_CUDA(cudaEventRecord(ev[2], st));
          FLZ_CUDA(cudaEventSynchronize(ev[2]));
        }
        P.S.push_back(S);
      }
    }
    if (tcb) tcb->check_status();
    if (fx) fx_check_flag(A);
    if (!keep) return;
    float a = 0.f, b = 0.f;
    FLZ_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
    FLZ_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
    ms_op += a;
    ms_orth += b;
  }

  // One block Lanczos step j: W = op(Q_j), reorthogonalize, QR into Q_{j+1}.
  void step(int j, const std::function<void(const T*, T*)>& op, Projected& P, double op_norm) {
    if (can_split()) {
      step_issue(j, op);
      step_finish(j, P, op_norm);
      return;
    }
    if (!ev[0])
      for (auto& x : ev) FLZ_CUDA(cudaEventCreate(&x));
    FLZ_CUDA(cudaEventRecord(ev[0], st));
    op(block(j), W);
    FLZ_CUDA(cudaEventRecord(ev[1], st));
    T* next = (j + 1 < nb_cap) ? block(j + 1) : nullptr;
    T* dst = next ? next : W;
    std::vector<double> D;
    cgs2(W, j + 1, &D);
    std::vector<double> S = block_qr(W, dst);
    P.D.push_back(D);
    // breakdown (as in step_finish)
    double smin = 1e300;
    for (int i = 0; i < r; ++i) smin = std::min(smin, std::fabs(S[i * r + i]));
    if (next && smin < 1e-12 * std::max(op_norm, 1e-300)) {
      cgs2(next, j + 1, nullptr);
      block_qr(next, next);
    }
    if (next) seal(j + 1);
    P.S.push_back(S);
    FLZ_CUDA(cudaEventRecord(ev[2], st));
    FLZ_CUDA(cudaEventSynchronize(ev[2]));
    if (tcb) tcb->check_status();
    if (fx) fx_check_flag(A);
    float a = 0.f, b = 0.f;
    FLZ_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
    FLZ_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
    ms_op += a;
    ms_orth += b;
  }
  ~Engine() {
    for (auto& x : ev)
      if (x) cudaEventDestroy(x);
  }
};

template <class T>
void orthonormal_start(Engine<T>& E, uint64_t seed) {
  random_normal(E.block(0), E.n * E.r, seed, 0, E.st);
  E.block_qr(E.block(0), E.block(0));
  E.seal(0);
}

// Warm start: r random combinations of the given start vectors (columns of
// the column-major X) plus noise of 1 % of their size, orthonormalized. A
// start block rich in the wanted eigenvectors (those of a nearby earlier
// problem) lets the filtered Krylov space reach them in fewer block steps; the
// noise keeps every direction present for eigenvectors that entered the window.
void warm_start(Engine<double>& E, const double* X, int cols, uint64_t seed) {
  const int r = E.r;
  const int64_t n = E.n;
  DevBuf<double> G;
  G.reserve((size_t)cols * r);
  random_normal(G.p, (int64_t)cols * r, seed ^ 0x77a7ull, 0, E.st);
  random_normal(E.block(0), n * r, seed, 0, E.st);
  // noise 0.01 / sqrt(n) per entry against combinations of unit columns (size ~ sqrt(cols / n))
  const double noise = 0.01 * std::sqrt((double)cols / (double)n);
  combine_columns(X, n, n, cols, G.p, r, noise, E.block(0), E.st);
  E.block_qr(E.block(0), E.block(0));
  E.seal(0);
}

// Spectrum bounds by block Lanczos on A (Section 2.2 after eq. transf).
void estimate_bounds(flz_matrix* A, int steps, int r, uint64_t seed, cudaStream_t st, double* lmin, double* lmax) {
  const int64_t n = A->n;
  // at least 15 block steps: with wide blocks a fixed vector count would leave
  // too low a Krylov degree to reach the extreme eigenvalues
  int nb = std::max(15, (steps + r - 1) / r);
  nb = (int)std::min<int64_t>(nb, std::max<int64_t>(1, n / r));
  DevBuf<double> Qb, Wb, Cb, C2b, partb, smallb;
  Qb.reserve((size_t)(nb + 1) * n * r);
  Wb.reserve((size_t)n * r);
  Cb.reserve((size_t)(nb + 1) * r * r);
  C2b.reserve((size_t)(nb + 1) * r * r);
  partb.reserve(std::max(basis_dot_scratch(n, nb + 1, r, r), (size_t)1));
  smallb.reserve((size_t)r * r);
  Engine<double> E{A, n, r, st, Qb.p, nb + 1, Wb.p, Cb.p, C2b.p, partb.p, smallb.p};
  orthonormal_start(E, seed ^ 0x5bd1e995ull);
  Projected P;
  P.r = r;
  const double anorm = std::max(std::fabs(A->glo), std::fabs(A->ghi));
  auto op = [&](const double* X, double* Y) { spmm(A, X, Y, r, r, st); };
  int k = 0;
  for (int j = 0; j < nb; ++j) {
    E.step(j, op, P, anorm);
    k = j + 1;
  }
  const int K = k * r;
  std::vector<double> T = P.assemble(k);
  std::vector<double> theta;
  band_eigenvalues(T, K, r, theta);
  std::vector<int> idx = {0, K - 1};
  std::vector<double> Y;
  band_eigenvectors(T, K, r, theta, idx, Y, seed);
  const std::vector<double>& S = P.S[k - 1];
  auto resbound = [&](int t) {
    // || S_k y_bottom ||
    const double* y = &Y[(size_t)t * K + (size_t)(k - 1) * r];
    double s2 = 0.0;
    for (int i = 0; i < r; ++i) {
      double v = 0.0;
      for (int a = 0; a < r; ++a) v += S[i * r + a] * y[a];
      s2 += v * v;
    }
    return std::sqrt(s2);
  };
  double lo = theta[0] - resbound(0);
  double hi = theta[K - 1] + resbound(1);
  // a tiny relative margin keeps the mapped extremes inside [-1, 1] under rounding
  const double margin = 1e-10 * std::max(1.0, hi - lo);
  lo -= margin;
  hi += margin;
  *lmin = std::max(lo, A->glo);
  *lmax = std::min(hi, A->ghi);
  if (!(*lmin < *lmax)) {
    *lmin = A->glo;
    *lmax = A->ghi;
  }
}

}  // namespace

void bounds_entry(flz_matrix* A, int steps, int r, uint64_t seed, cudaStream_t st, double* lmin, double* lmax) {
  estimate_bounds(A, steps, r, seed, st, lmin, lmax);
}

namespace {

// W = p_m(Ahat) X on the engine's storage type.
void apply_filter(flz_matrix* A, double c, double e, const std::vector<double>& coeffs, int m, int r,
                  const flz_params& p, const double* X, double* Y, cudaStream_t st) {
  filter_apply(A, c, e, coeffs.data(), m, r, X, Y, p.precision, p.recurrence, st);
}
void apply_filter(flz_matrix* A, double c, double e, const std::vector<double>& coeffs, int m, int r,
                  const flz_params& p, const dev::dfloat* X, dev::dfloat* Y, cudaStream_t st) {
  filter_apply(A, c, e, coeffs.data(), m, r, X, Y, p.recurrence, st);
}

// The in-window pairs of a subspace sweep's block (rr over Xr, blocks of 16
// rows-major columns) become the solver's eigenvectors, as unit columns.
void store_refined(flz_solver* s, const RefineResult& rr, const double* Xr, cudaStream_t st) {
  const int64_t n = s->A->n;
  const int64_t found = (int64_t)rr.vals.size();
  s->evecs.reserve((size_t)std::max<int64_t>(found, 1) * n);
  for (int64_t i = 0; i < found; ++i) {
    const int col = rr.index[i];
    rows_to_columns(Xr + (size_t)(col / 16) * n * 16 + (col % 16), n, 1, 16, s->evecs.p + (size_t)i * n, n, st);
  }
  DevBuf<double> dv, prt;
  dv.reserve(2);
  prt.reserve(column_sums_scratch(n, 1) + 64);
  for (int64_t i = 0; i < found; ++i) {
    double* x = s->evecs.p + (size_t)i * n;
    column_sums(x, x, nullptr, n, 1, 1, 0, dv.p, prt.p, st);
    double xx = 0.0;
    FLZ_CUDA(cudaMemcpyAsync(&xx, dv.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    const double sc = 1.0 / std::sqrt(std::max(xx, 1e-300));
    FLZ_CUDA(cudaMemcpyAsync(dv.p + 1, &sc, sizeof(double), cudaMemcpyHostToDevice, st));
    basis_update(x, 1, n, 1, dv.p + 1, 1, 1.0, 0.0, x, 1, st);
  }
  FLZ_CUDA(cudaStreamSynchronize(st));
}

// Sorts the found pairs ascending (eigenvectors with them) into the solver's results.
void finish_results(flz_solver* s, const std::vector<double>& found_vals, const std::vector<double>& found_res,
                    cudaStream_t st) {
  const int64_t n = s->A->n;
  const int found = (int)found_vals.size();
  std::vector<int> perm(found);
  for (int i = 0; i < found; ++i) perm[i] = i;
  std::sort(perm.begin(), perm.end(), [&](int a, int b) { return found_vals[a] < found_vals[b]; });
  bool sorted = true;
  for (int i = 0; i < found; ++i) sorted &= perm[i] == i;
  if (!sorted && found > 0) {
    DevBuf<double> tmp;
    tmp.reserve((size_t)found * n);
    for (int i = 0; i < found; ++i)
      FLZ_CUDA(cudaMemcpyAsync(tmp.p + (size_t)i * n, s->evecs.p + (size_t)perm[i] * n, sizeof(double) * n,
                               cudaMemcpyDeviceToDevice, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    std::swap(tmp.p, s->evecs.p);
    std::swap(tmp.count, s->evecs.count);
  }
  s->evals.resize(found);
  s->resid.resize(found);
  double maxres = 0.0;
  for (int i = 0; i < found; ++i) {
    s->evals[i] = found_vals[perm[i]];
    s->resid[i] = found_res[perm[i]];
    maxres = std::max(maxres, s->resid[i]);
  }
  s->count = found;
  s->solved = true;
  s->stats.count = found;
  s->stats.max_residual = maxres;
}

template <class BT>
flz_status solve_impl(flz_solver* s, cudaStream_t st) {
  const auto t_start = Clock::now();
  const int64_t launches0 = g_kernel_launches;
  flz_matrix* A = s->A;
  const flz_params& p = s->p;
  const int64_t n = A->n;
  const int r = p.block_size;
  flz_stats& stats = s->stats;
  stats = flz_stats{};
  stats.block_size = r;
  s->checks.clear();
  s->solved = false;
  s->count = 0;
  s->evals.clear();
  s->resid.clear();
  if (r < 1 || r > 16 || r > n) fail(FLZ_ERR_INVALID_ARG, "block size %d invalid for n = %lld", r, (long long)n);

  // 1. bounds
  auto t0 = Clock::now();
  double lmin, lmax;
  if (p.lmin < p.lmax) {
    lmin = p.lmin;
    lmax = p.lmax;
  } else {
    estimate_bounds(A, p.bounds_steps, r, p.seed * 7919u + 17u, st, &lmin, &lmax);
  }
  stats.ms_bounds = ms_since(t0);
  // The Gershgorin interval contains the spectrum: an interval outside it is
  // empty. One inside it but outside the Lanczos estimate means the estimate
  // missed an extreme eigenvalue; the estimate is widened to cover it.
  if (s->beta < A->glo || s->alpha > A->ghi)
    fail(FLZ_ERR_EMPTY_INTERVAL, "[%g, %g] misses the Gershgorin interval [%g, %g]", s->alpha, s->beta, A->glo, A->ghi);
  if (s->beta < lmin) lmin = std::max(s->alpha, A->glo);
  if (s->alpha > lmax) lmax = std::min(s->beta, A->ghi);
  if (!(lmax > lmin)) {  // a single-point spectrum (n = 1, A = cI): any enclosing interval maps it
    const double pad = 1e-3 * std::max(1.0, std::fabs(lmin));
    lmin -= pad;
    lmax += pad;
  }
  stats.lmin = lmin;
  stats.lmax = lmax;
  // 2. map (eq. transf)
  const double c = 0.5 * (lmin + lmax), e = 0.5 * (lmax - lmin);
  stats.c = c;
  stats.e = e;
  double am = (s->alpha - c) / e, bm = (s->beta - c) / e;
  if (bm < -1.0 || am > 1.0) fail(FLZ_ERR_EMPTY_INTERVAL, "[%g, %g] misses the spectrum [%g, %g]", s->alpha, s->beta, lmin, lmax);
  am = std::max(am, -1.0);
  bm = std::min(bm, 1.0);
  stats.alpha_mapped = am;
  stats.beta_mapped = bm;
  // 3. degree and coefficients. A window that covers the whole mapped
  // spectrum makes the filter constant (p = 1), which separates nothing in
  // the Rayleigh-Ritz step on p(A); it runs unfiltered block Lanczos instead
  // (the degree-1 operator p(z) = z, whose Ritz values are monotone in lambda).
  const bool whole = am <= -1.0 && bm >= 1.0;
  const int m = whole ? 1 : (p.degree > 0 ? p.degree : auto_degree(am, bm, p.degree_eps, p.max_degree));
  if (m < 0) fail(FLZ_ERR_CAPACITY, "no degree <= %d meets the degree rule", p.max_degree);
  stats.degree = m;
  std::vector<double> coeffs(m + 1);
  if (whole) {
    coeffs[0] = 0.0;
    coeffs[1] = 1.0;
  } else {
    filter_coeffs_for(p, am, bm, m, coeffs.data());
  }
  const double anorm = std::max(std::fabs(lmin), std::fabs(lmax));
  const int guard = p.guard > 0 ? p.guard : std::max(r, 3);

  // 3b. subspace start (params.start_mode SUBSPACE): filtered subspace
  // iteration on [start vectors, guard and extra columns]; on success the
  // solve ends here, without a Krylov basis.
  if constexpr (std::is_same<BT, double>::value)
    if (s->start_cols > 0 && p.start_mode == FLZ_START_SUBSPACE && !whole) {
      int kp = s->start_cols + guard + std::max(16, s->start_cols / 3);
      kp = (kp + 15) / 16 * 16;
      if ((int64_t)kp * 4 <= n) {
        DevBuf<double> Xr;
        Xr.reserve((size_t)n * kp);
        random_normal(Xr.p, n * kp, p.seed ^ 0x5eed5ull, 0, st);
        columns_to_blocks(s->start.p, n, n, s->start_cols, Xr.p, st);
        std::vector<double> half;
        if (m >= 8) {
          half.resize(m / 2 + 1);
          filter_coeffs_for(p, am, bm, m / 2, half.data());
        }
        RefineArgs ra{s->alpha, s->beta, lmin, lmax, p.tol, 12, std::max(m, 64), coeffs, half, s->start_cols};
        ra.flat_first = true;
        ra.stop_on_stall = true;
        // After Rayleigh-Ritz a Ritz vector's error lies outside the block's
        // span, so a steep damping polynomial (up to the 1e6 cap across the
        // window) cannot let the favoured pairs swamp the others.
        ra.range_scale = 1e30;
        // about what filtered Lanczos would take: three block vectors per
        // wanted or guard pair, each at the solve's degree
        ra.matvec_budget = 3 * (int64_t)(s->start_cols + guard) * m;
        RefineResult rr;
        bool ok = false;
        try {
          rr = refine(A, ra, Xr.p, kp, st);
          ok = rr.converged && rr.outside >= guard;
        } catch (const Failure& f) {
          if (f.status != FLZ_ERR_NOT_CONVERGED) throw;  // a lost rank falls back; device errors do not
          clear_last_error();
        }
        stats.refine_sweeps = rr.sweeps;
        stats.refine_degree = rr.degrees.empty() ? 0 : *std::max_element(rr.degrees.begin(), rr.degrees.end());
        stats.ms_refine = rr.ms;
        stats.sweep_matvecs = rr.matvecs;
        if (ok) {
          store_refined(s, rr, Xr.p, st);
          finish_results(s, rr.vals, rr.res, st);
          stats.start_used = 2;
          stats.converged = 1;
          stats.ms_total = ms_since(t_start);
          stats.kernel_launches = g_kernel_launches - launches0;
          stats.filter_precision = A->last_filter_precision;
          return FLZ_OK;
        }
      }
    }

  // 4. basis capacity
  int64_t kcap = p.max_basis > 0 ? p.max_basis : 2000;
  kcap = std::min<int64_t>(kcap, n);
  size_t free_b = 0, total_b = 0;
  FLZ_CUDA(cudaMemGetInfo(&free_b, &total_b));
  // Reorthogonalization on the tensor cores where it applies; AUTO keeps the
  // FP64 pipes when the digit copy (16 bytes per value) would shrink the basis.
  bool use_tc = false;
  if constexpr (std::is_same<BT, double>::value)
    use_tc = p.ortho == FLZ_ORTHO_TENSOR || (p.ortho == FLZ_ORTHO_AUTO && TcBasis::supported(r));
  if (use_tc) {
    // the FP64 basis and its digit copy (24 bytes per value) may take 3/4 of the free memory
    const double budget = 0.75 * (double)free_b + (double)s->tcb.q.count;
    const int64_t tc_cap =
        (int64_t)(budget / (8.0 * (double)n + (double)TcBasis::bytes_for(n, 16) / 16.0));
    if (p.ortho == FLZ_ORTHO_AUTO && tc_cap < kcap)
      use_tc = false;
    else
      kcap = std::min(kcap, std::max<int64_t>(tc_cap, 2 * r));
  }
  if (!use_tc) {
    s->tcb.release();
    const int64_t mem_cap = (int64_t)(0.6 * (double)free_b / (8.0 * (double)n));
    kcap = std::min(kcap, std::max<int64_t>(mem_cap, 2 * r));
  }
  stats.ortho = use_tc ? FLZ_ORTHO_TENSOR : FLZ_ORTHO_CUDA_CORES;
  const int nb_cap = (int)std::max<int64_t>(2, kcap / r);
  s->Q.reserve((size_t)nb_cap * n * r);
  s->W.reserve((size_t)n * r);
  s->C.reserve((size_t)nb_cap * r * r);
  s->C2.reserve((size_t)nb_cap * r * r);
  s->part.reserve(std::max(basis_dot_scratch(n, nb_cap, r, r), (size_t)1));
  s->small.reserve(16 * 16 + 64 + qr_device_scratch());  // host-path R^{-1}; the device QR's scratch after it
  s->X.reserve((size_t)n * 16);
  s->AX.reserve((size_t)n * 16);
  FLZ_CUDA(cudaMemsetAsync(s->X.p, 0, sizeof(double) * n * 16, st));  // columns a short chunk leaves unwritten
  s->colpart.reserve(column_sums_scratch(n, 16) + 64);
  static_assert(sizeof(BT) == sizeof(double), "basis storage reuses the FP64 buffers");
  BT* Qt = reinterpret_cast<BT*>(s->Q.p);
  Engine<BT> E{A, n, r, st, Qt, nb_cap, reinterpret_cast<BT*>(s->W.p), s->C.p, s->C2.p, s->part.p, s->small.p};
  if constexpr (std::is_same<BT, double>::value) {
    if (!s->pinned) FLZ_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s->pinned), sizeof(double) * 3 * 16 * 16));
    E.pinned = s->pinned;
    E.qrs = s->small.p + 16 * 16 + 64;
  }
  if (use_tc) {
    s->tcb.reserve(n, (int64_t)nb_cap * r);
    E.tcb = &s->tcb;
  }
  E.fx = p.precision == FLZ_PREC_FX64;
  bool warm = false;
  if constexpr (std::is_same<BT, double>::value)
    if (s->start_cols > 0) {
      warm_start(E, s->start.p, s->start_cols, p.seed);
      warm = true;
      stats.start_used = 1;
    }
  if (!warm) orthonormal_start(E, p.seed);

  Projected P;
  P.r = r;
  auto filt = [&](const BT* X, BT* Y) { apply_filter(A, c, e, coeffs, m, r, p, X, Y, st); };
  double ms_check = 0.0;
  int64_t prev_count = -1;
  bool converged = false;
  int k = 0;
  // Pairs the last walk visited: the next check first requires at least this
  // many leading Ritz pairs to pass the cheap p(A) residual gate.
  int gate_len = 16;
  // If x has ||Ax - lambda x|| <= tol ||A|| then ||p(A)x - theta x|| <=
  // max|p'| tol ||A|| / e, and max|p'| <= 1.1 m^2 on [-1, 1] (Markov, |p| <= 1.1):
  // a pair whose p(A) residual exceeds this cannot pass the A-residual test.
  // With refinement (reduced-precision filter) the filtered Lanczos phase stops
  // at the filter's floor and the refinement brings the pairs to p.tol.
  const bool refining = p.refine == 1 && (p.precision == FLZ_PREC_FP32 || p.precision == FLZ_PREC_BF16);
  const double tol = refining ? std::max(p.tol, p.precision == FLZ_PREC_FP32 ? 1e-5 : 1e-2) : p.tol;
  const double p_gate = std::min(1e-2, 10.0 * 1.1 * (double)m * m * tol * anorm / e);
  std::vector<double> found_vals, found_res;
  std::vector<double> lastT, lastTheta;  // the last check's T_k and its eigenvalues (refinement)
  int64_t found = 0;
  for (int j = 0; j < nb_cap; ++j) {
    if (E.issued) E.step_finish(j, P, 1.0);  // issued before the previous check's host work
    else E.step(j, filt, P, 1.0);
    k = j + 1;
    const bool last = (k == nb_cap) || ((int64_t)(k + 1) * r > n);
    if (k % p.check_every != 0 && !last) continue;
    // the next block step runs on the GPU while the host works on this check
    // (its results are dropped if the check ends the solve); the check's GPU
    // work queues behind it and reads only the first k blocks
    if (E.can_split() && !last) E.step_issue(j + 1, filt);

    // ---- convergence check ----
    const auto tc = Clock::now();
    stats.checks++;
    const int K = k * r;
    std::vector<double> T = P.assemble(k);
    std::vector<double> theta;
    band_eigenvalues(T, K, r, theta);
    std::vector<int> order(K);
    for (int i = 0; i < K; ++i) order[i] = K - 1 - i;  // descending theta
    const std::vector<double>& Sk = P.S[k - 1];
    int inside = 0, outside = 0;
    bool all_small = true, walk_done = false;
    found_vals.clear();
    found_res.clear();
    found = 0;
    auto p_residual = [&](const double* y) {  // ||S_k y_bottom|| of a unit eigenvector y of T_k
      double s2 = 0.0;
      for (int i = 0; i < r; ++i) {
        double v = 0.0;
        for (int a = 0; a < r; ++a) v += Sk[i * r + a] * y[(size_t)(k - 1) * r + a];
        s2 += v * v;
      }
      return std::sqrt(s2);
    };
    {
      // cheap host gate: the leading gate_len pairs must all pass before any GPU work
      // in batches of 8 from the largest theta down, stopping at the first failure
      const int g_cnt = std::min(gate_len, K);
      for (int g0 = 0; g0 < g_cnt && all_small; g0 += 8) {
        std::vector<int> gidx(order.begin() + g0, order.begin() + std::min(g_cnt, g0 + 8));
        std::vector<double> Yg;
        band_eigenvectors(T, K, r, theta, gidx, Yg, p.seed + (uint64_t)g0);
        for (size_t t = 0; t < gidx.size() && all_small; ++t)
          if (!(p_residual(&Yg[t * K]) <= p_gate)) all_small = false;
      }
    }
    int walked = 0;
    std::vector<double> walkY;  // eigenvectors of T formed so far in this check
    std::vector<int> walkIdx;
    for (int pos = 0; pos < K && !walk_done && all_small; pos += 16) {
      const int cnt = std::min(16, K - pos);
      // eigenvectors of T for this chunk, kept orthogonal to the earlier
      // chunks' vectors of nearby eigenvalues (copies of a multiple
      // eigenvalue may straddle two chunks)
      std::vector<int> idx(order.begin() + pos, order.begin() + pos + cnt);
      std::vector<double> Y;
      band_eigenvectors(T, K, r, theta, idx, Y, p.seed, &walkY, &walkIdx);
      walkY.insert(walkY.end(), Y.begin(), Y.end());
      walkIdx.insert(walkIdx.end(), idx.begin(), idx.end());
      // a pair failing the gate ends the walk before its Ritz vector is formed
      if (!(p_residual(&Y[0]) <= p_gate)) {
        all_small = false;
        break;
      }
      // Ritz vectors X = Q_k Y (n x 16, zero-padded columns)
      std::vector<double> Cy((size_t)K * 16, 0.0);
      for (int t = 0; t < cnt; ++t)
        for (int i = 0; i < K; ++i) Cy[(size_t)i * 16 + t] = Y[(size_t)t * K + i];
      s->C2.reserve(std::max(s->C2.count, (size_t)K * 16));
      E.C2 = s->C2.p;
      FLZ_CUDA(cudaMemcpyAsync(s->C2.p, Cy.data(), sizeof(double) * K * 16, cudaMemcpyHostToDevice, st));
      bool tc_ritz = false;
      if constexpr (std::is_same<BT, double>::value)
        if (E.tcb) {
          E.tcb->multiply(K, s->C2.p, 16, cnt, s->X.p, 16, st);
          tc_ritz = true;
        }
      if (!tc_ritz) basis_update(Qt, k, n, r, s->C2.p, 16, 1.0, 0.0, s->X.p, 16, st);
      spmm(A, s->X.p, s->AX.p, 16, 16, st);
      double* dev = s->small.p;  // [0,16) xx, [16,32) xAx, [32,48) lam, [48,64) res2, [64] scale
      column_sums(s->X.p, s->X.p, nullptr, n, 16, 16, 0, dev, s->colpart.p, st);
      column_sums(s->X.p, s->AX.p, nullptr, n, 16, 16, 0, dev + 16, s->colpart.p, st);
      double h[64];
      FLZ_CUDA(cudaMemcpyAsync(h, dev, sizeof(double) * 32, cudaMemcpyDeviceToHost, st));
      FLZ_CUDA(cudaStreamSynchronize(st));
      for (int t = 0; t < 16; ++t) h[32 + t] = (t < cnt && h[t] > 0) ? h[16 + t] / h[t] : 0.0;
      FLZ_CUDA(cudaMemcpyAsync(dev + 32, h + 32, sizeof(double) * 16, cudaMemcpyHostToDevice, st));
      column_sums(s->X.p, s->AX.p, dev + 32, n, 16, 16, 1, dev + 48, s->colpart.p, st);
      FLZ_CUDA(cudaMemcpyAsync(h + 48, dev + 48, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
      FLZ_CUDA(cudaStreamSynchronize(st));
      for (int t = 0; t < cnt; ++t) {
        ++walked;
        const double xx = h[t];
        const double lam = h[32 + t];
        const double res = std::sqrt(std::max(h[48 + t], 0.0) / std::max(xx, 1e-300)) / anorm;
        if (!(res <= tol)) {
          all_small = false;
          walk_done = true;
          break;
        }
        if (lam >= s->alpha && lam <= s->beta) {
          // keep x / ||x|| as a result column
          const size_t need = (size_t)(found + 1) * n;
          if (s->evecs.count < need) {
            DevBuf<double> grown;
            grown.reserve(std::max(need, s->evecs.count * 2));
            if (found > 0)
              FLZ_CUDA(cudaMemcpyAsync(grown.p, s->evecs.p, sizeof(double) * found * n, cudaMemcpyDeviceToDevice, st));
            std::swap(grown.p, s->evecs.p);
            std::swap(grown.count, s->evecs.count);
          }
          rows_to_columns(s->X.p + t, n, 1, 16, s->evecs.p + (size_t)found * n, n, st, 1.0 / std::sqrt(xx));
          found_vals.push_back(lam);
          found_res.push_back(res);
          ++found;
          ++inside;
        } else {
          ++outside;
          if (outside >= guard) {
            walk_done = true;
            break;
          }
        }
      }
      if (!walk_done && pos + cnt >= K) walk_done = true;
    }
    if (walked > 0) gate_len = std::max(16, walked);
    // A basis spanning the whole space (K = n) whose every Ritz pair passed
    // holds all eigenpairs: no guard pairs outside the interval need exist
    // (a window covering the whole spectrum, tiny matrices).
    const bool full_space = walked == K && (int64_t)K >= n;
    const bool complete = all_small && (outside >= guard || full_space);
    converged = complete && (full_space || (prev_count >= 0 && inside == prev_count));
    prev_count = complete ? inside : -1;
    s->checks.push_back(flz_check{(int64_t)k, (int64_t)inside, walked, outside, all_small ? 1 : 0, converged ? 1 : 0});
    ms_check += ms_since(tc);
    if (refining && (converged || last)) {
      lastT.swap(T);
      lastTheta.swap(theta);
    }
    if (converged || last) {
      if (E.issued) E.step_finish(k, P, 1.0, false);
      break;
    }
  }
  FLZ_CUDA(cudaStreamSynchronize(st));
  if (E.tcb) {  // the last check's Ritz vectors ran after the last step's status read
    FLZ_CUDA(cudaMemcpy(E.tcb->status_host, E.tcb->status.p, sizeof(int), cudaMemcpyDeviceToHost));
    E.tcb->check_status();
  }
  if constexpr (std::is_same<BT, double>::value)
    if (refining && converged && !lastT.empty()) {
      // Ritz vectors of the leading kp pairs by p(A) Ritz value: the wanted and
      // guard pairs and as many again as a third of the wanted (at least 16),
      // in whole blocks of 16 columns
      const int K = k * r;
      int kp = (int)(found + guard + std::max<int64_t>(16, found / 3));
      kp = std::min((kp + 15) / 16 * 16, K / 16 * 16);
      if (kp >= 16) {
        std::vector<int> idx(kp);
        for (int i = 0; i < kp; ++i) idx[i] = K - 1 - i;  // descending theta
        std::vector<double> Yt;
        band_eigenvectors(lastT, K, r, lastTheta, idx, Yt, p.seed);
        DevBuf<double> Xr, Cb;
        Xr.reserve((size_t)n * kp);
        Cb.reserve((size_t)K * 16);
        std::vector<double> hc((size_t)K * 16);
        for (int b = 0; b < kp / 16; ++b) {
          for (int t = 0; t < 16; ++t)
            for (int i = 0; i < K; ++i) hc[(size_t)i * 16 + t] = Yt[(size_t)(16 * b + t) * K + i];
          FLZ_CUDA(cudaMemcpyAsync(Cb.p, hc.data(), sizeof(double) * K * 16, cudaMemcpyHostToDevice, st));
          if (E.tcb)
            E.tcb->multiply(K, Cb.p, 16, 16, Xr.p + (size_t)b * n * 16, 16, st);
          else
            basis_update(Qt, k, n, r, Cb.p, 16, 1.0, 0.0, Xr.p + (size_t)b * n * 16, 16, st);
          FLZ_CUDA(cudaStreamSynchronize(st));  // hc is reused for the next block
        }
        std::vector<double> half;
        if (!whole && m >= 8) {
          half.resize(m / 2 + 1);
          filter_coeffs_for(p, am, bm, m / 2, half.data());
        }
        RefineArgs ra{s->alpha, s->beta, lmin, lmax, p.tol, p.precision == FLZ_PREC_FP32 ? 4 : 10,
                      std::max(m, 64), coeffs, half, (int)found};
        const RefineResult rr = refine(A, ra, Xr.p, kp, st);
        stats.refine_sweeps = rr.sweeps;
        stats.refine_degree = rr.degrees.empty() ? 0 : *std::max_element(rr.degrees.begin(), rr.degrees.end());
        stats.ms_refine = rr.ms;
        converged = rr.converged;
        found = (int64_t)rr.vals.size();
        found_vals = rr.vals;
        found_res = rr.res;
        stats.sweep_matvecs = rr.matvecs;
        store_refined(s, rr, Xr.p, st);
      }
    }

  finish_results(s, found_vals, found_res, st);
  stats.iters = k;
  stats.matvecs = (int64_t)r * m * k;
  stats.converged = converged ? 1 : 0;
  stats.ms_filter = E.ms_op;
  stats.ms_orth = E.ms_orth;
  stats.ms_check = ms_check;
  stats.basis_vectors = (int64_t)k * r;
  stats.ms_total = ms_since(t_start);
  stats.kernel_launches = g_kernel_launches - launches0;
  stats.filter_precision = A->last_filter_precision;
  return converged ? FLZ_OK : FLZ_ERR_NOT_CONVERGED;
}

}  // namespace

// The double-FP32 precision keeps the whole Krylov basis as double-FP32
// pairs: filter, reorthogonalization and block QR run on the FP32 pipes;
// Rayleigh-Ritz, Rayleigh quotients and residuals stay FP64.
flz_status solve(flz_solver* s, cudaStream_t st) {
  if (s->p.precision == FLZ_PREC_DF64) return solve_impl<dev::dfloat>(s, st);
  return solve_impl<double>(s, st);
}

// Spectrum slicing (named as future work in Section 5): [alpha, beta] is cut
// into `nslices` equal-width sub-intervals solved one after another on the
// same matrix with the same bounds (estimated once), each with its own
// smaller Krylov basis. A pair found by two adjacent slices (an eigenvalue
// on a shared endpoint) is kept once: two results count as the same pair
// when their eigenvalues agree to 10 tol ||A|| and their eigenvectors
// overlap by more than 1/2; the one with the smaller residual stays.
flz_status solve_sliced(flz_solver* s, int nslices, cudaStream_t st) {
  if (nslices < 1) fail(FLZ_ERR_INVALID_ARG, "nslices must be >= 1");
  if (nslices == 1) return solve(s, st);
  const auto t_start = Clock::now();
  flz_matrix* A = s->A;
  const int64_t n = A->n;
  const flz_params& p = s->p;
  if (p.block_size < 1 || p.block_size > 16 || p.block_size > n) fail(FLZ_ERR_INVALID_ARG, "block size invalid");
  s->solved = false;
  s->count = 0;
  s->evals.clear();
  s->resid.clear();
  double lmin, lmax;
  const auto tb = Clock::now();
  if (p.lmin < p.lmax) {
    lmin = p.lmin;
    lmax = p.lmax;
  } else {
    estimate_bounds(A, p.bounds_steps, p.block_size, p.seed * 7919u + 17u, st, &lmin, &lmax);
  }
  const double ms_bounds = ms_since(tb);
  if (s->beta < A->glo || s->alpha > A->ghi)
    fail(FLZ_ERR_EMPTY_INTERVAL, "[%g, %g] misses the Gershgorin interval [%g, %g]", s->alpha, s->beta, A->glo, A->ghi);
  if (s->beta < lmin) lmin = std::max(s->alpha, A->glo);
  if (s->alpha > lmax) lmax = std::min(s->beta, A->ghi);
  if (!(lmax > lmin)) {
    const double pad = 1e-3 * std::max(1.0, std::fabs(lmin));
    lmin -= pad;
    lmax += pad;
  }
  const double lo = std::max(s->alpha, lmin), hi = std::min(s->beta, lmax);
  const double anorm = std::max(std::fabs(lmin), std::fabs(lmax));

  flz_solver sub;
  sub.A = A;
  sub.p = p;
  sub.p.lmin = lmin;
  sub.p.lmax = lmax;
  sub.has_interval = true;
  std::vector<double> vals, res;
  std::vector<int> slice_of;
  DevBuf<double> vecs;  // n x total, column-major
  flz_stats agg{};
  agg.block_size = p.block_size;
  agg.lmin = lmin;
  agg.lmax = lmax;
  agg.converged = 1;
  bool all_ok = true;
  for (int i = 0; i < nslices; ++i) {
    sub.alpha = lo + (hi - lo) * i / nslices;
    sub.beta = (i + 1 == nslices) ? hi : lo + (hi - lo) * (i + 1) / nslices;
    sub.p.seed = p.seed + 104729ull * (uint64_t)i;
    const flz_status si = solve(&sub, st);
    if (si != FLZ_OK) all_ok = false;
    const int64_t c = sub.count;
    if (c > 0) {
      const size_t have = vals.size();
      DevBuf<double> grown;
      grown.reserve((have + c) * (size_t)n);
      if (have > 0) FLZ_CUDA(cudaMemcpyAsync(grown.p, vecs.p, sizeof(double) * have * n, cudaMemcpyDeviceToDevice, st));
      FLZ_CUDA(cudaMemcpyAsync(grown.p + have * n, sub.evecs.p, sizeof(double) * c * n, cudaMemcpyDeviceToDevice, st));
      FLZ_CUDA(cudaStreamSynchronize(st));
      std::swap(grown.p, vecs.p);
      std::swap(grown.count, vecs.count);
      for (int64_t j = 0; j < c; ++j) {
        vals.push_back(sub.evals[j]);
        res.push_back(sub.resid[j]);
        slice_of.push_back(i);
      }
    }
    const flz_stats& x = sub.stats;
    agg.iters += x.iters;
    agg.matvecs += x.matvecs;
    agg.degree = std::max(agg.degree, x.degree);
    agg.checks += x.checks;
    agg.converged = agg.converged && x.converged;
    agg.ms_filter += x.ms_filter;
    agg.ms_orth += x.ms_orth;
    agg.ms_check += x.ms_check;
    agg.basis_vectors = std::max(agg.basis_vectors, x.basis_vectors);
    agg.kernel_launches += x.kernel_launches;
    agg.max_residual = std::max(agg.max_residual, x.max_residual);
    agg.ortho = x.ortho;
    agg.filter_precision = x.filter_precision;
  }
  // merge: ascending order, pairs shared by adjacent slices kept once
  const int64_t total = (int64_t)vals.size();
  std::vector<int> order(total);
  for (int64_t i = 0; i < total; ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return vals[a] < vals[b]; });
  std::vector<char> drop(total, 0);
  DevBuf<double> part, out1;
  part.reserve(column_sums_scratch(n, 1) + 64);
  out1.reserve(1);
  auto overlap = [&](int ia, int ib) {
    column_sums(vecs.p + (size_t)ia * n, vecs.p + (size_t)ib * n, nullptr, n, 1, 1, 0, out1.p, part.p, st);
    double ov = 0.0;
    FLZ_CUDA(cudaMemcpyAsync(&ov, out1.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    return ov;
  };
  // clusters of eigenvalues that agree to 10 tol ||A||: when one holds results
  // of several slices, the slice with the most members is kept whole; a result
  // of another slice is dropped if its eigenvector lies mostly in the span of
  // the kept ones (a repeated copy, possibly rotated inside a multiple
  // eigenspace), and otherwise kept after orthogonalization against them
  // (its Rayleigh quotient and residual recomputed): the two slices may each
  // hold a different vector of one multiple eigenspace whose Rayleigh
  // quotients fall on either side of the shared endpoint.
  DevBuf<double> ax, scal;
  ax.reserve((size_t)n);
  scal.reserve(4);
  auto put = [&](double v) {
    FLZ_CUDA(cudaMemcpyAsync(scal.p, &v, sizeof(double), cudaMemcpyHostToDevice, st));
  };
  auto refresh = [&](int m) {  // unit-normalize vector m; recompute its Rayleigh quotient and residual
    double* x = vecs.p + (size_t)m * n;
    const double nrm = std::sqrt(std::max(overlap(m, m), 1e-300));
    put(1.0 / nrm);
    basis_update(x, 1, n, 1, scal.p, 1, 1.0, 0.0, x, 1, st);
    spmm(A, x, ax.p, 1, 1, st);
    column_sums(x, ax.p, nullptr, n, 1, 1, 0, out1.p, part.p, st);
    double lam = 0.0;
    FLZ_CUDA(cudaMemcpyAsync(&lam, out1.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    put(lam);
    column_sums(x, ax.p, scal.p, n, 1, 1, 1, out1.p, part.p, st);
    double r2 = 0.0;
    FLZ_CUDA(cudaMemcpyAsync(&r2, out1.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    vals[m] = lam;
    res[m] = std::sqrt(std::max(r2, 0.0)) / anorm;
  };
  const double close = 10.0 * p.tol * anorm;
  for (int64_t a = 0; a < total;) {
    int64_t b = a + 1;
    while (b < total && vals[order[b]] - vals[order[b - 1]] <= close) ++b;
    std::vector<int> members(order.begin() + a, order.begin() + b);
    std::vector<int> per_slice(nslices, 0);
    for (int m : members) per_slice[slice_of[m]]++;
    int primary = 0;
    for (int i = 1; i < nslices; ++i)
      if (per_slice[i] > per_slice[primary]) primary = i;
    int slices_present = 0;
    for (int i = 0; i < nslices; ++i) slices_present += per_slice[i] > 0;
    if (slices_present > 1) {
      std::vector<int> kept;
      for (int m : members)
        if (slice_of[m] == primary) kept.push_back(m);
      for (int m : members) {
        if (slice_of[m] == primary) continue;
        std::vector<double> ovs;
        double proj2 = 0.0;
        for (int u : kept) {
          ovs.push_back(overlap(m, u));
          proj2 += ovs.back() * ovs.back();
        }
        if (proj2 > 0.5) {
          drop[m] = 1;
          continue;
        }
        double* x = vecs.p + (size_t)m * n;
        for (int pass = 0; pass < 2; ++pass) {  // Gram-Schmidt twice against the kept vectors
          for (size_t q = 0; q < kept.size(); ++q) {
            const double ov = pass == 0 ? ovs[q] : overlap(m, kept[q]);
            put(-ov);
            basis_update(vecs.p + (size_t)kept[q] * n, 1, n, 1, scal.p, 1, 1.0, 1.0, x, 1, st);
          }
        }
        refresh(m);
        kept.push_back(m);
      }
    }
    a = b;
  }
  // the refreshed Rayleigh quotients may reorder neighbours
  std::sort(order.begin(), order.end(), [&](int x, int y) { return vals[x] < vals[y]; });
  std::vector<int> keep;
  for (int64_t a = 0; a < total; ++a)
    if (!drop[order[a]]) keep.push_back(order[a]);
  const int64_t found = (int64_t)keep.size();
  s->evecs.reserve((size_t)std::max<int64_t>(found, 1) * n);
  s->evals.resize(found);
  s->resid.resize(found);
  for (int64_t i = 0; i < found; ++i) {
    FLZ_CUDA(cudaMemcpyAsync(s->evecs.p + (size_t)i * n, vecs.p + (size_t)keep[i] * n, sizeof(double) * n,
                             cudaMemcpyDeviceToDevice, st));
    s->evals[i] = vals[keep[i]];
    s->resid[i] = res[keep[i]];
  }
  FLZ_CUDA(cudaStreamSynchronize(st));
  s->count = found;
  s->solved = true;
  agg.count = found;
  agg.ms_bounds = ms_bounds;
  agg.c = 0.5 * (lmin + lmax);
  agg.e = 0.5 * (lmax - lmin);
  agg.ms_total = ms_since(t_start);
  s->stats = agg;
  return all_ok ? FLZ_OK : FLZ_ERR_NOT_CONVERGED;
}

}  // namespace flz
