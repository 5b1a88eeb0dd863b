// Refinement of a reduced-precision solve (the mixed-precision form; not in
// the paper, which is FP64 throughout).
//
// With the filter in FP32 or BF16 storage the filtered Lanczos relation holds
// only to that rounding, and so does the Krylov basis: the Ritz vectors stall
// with errors of that size spread over the whole spectrum (residuals near
// 1e-7 in FP32). Their errors are removed by filtered subspace iteration in
// FP64-class arithmetic on the block [wanted pairs, guard pairs, extra pairs]:
//
//   sweep:  Y = p(Ahat) X                  (the 64-bit fixed-point filter,
//                                           or FP64 where it does not apply)
//           M = Y^T Y,  H = Y^T A Y        (exact digit products on the
//                                           tensor cores, FP64 results)
//           H v = mu M v                   (host, FP64)
//           X = Y V,  residuals ||A x - mu x|| / ||A||  (Section 2.3's
//                                           Rayleigh-Ritz, here on A itself)
//
// The filter damps everything above (for a window at the bottom of the
// spectrum; below it for one at the top) the largest Rayleigh quotient of
// the block: a Chebyshev polynomial T_d of that damping interval, rescaled to
// be at most 1 in magnitude on the whole spectrum (so the fixed-point kernel
// can evaluate it). Its degree is the largest whose ratio of values across the
// window stays below 0.01 / (the current residual): a larger ratio would let
// the small errors of the pairs it favours swamp the pairs it does not. The
// extra pairs push the block past the window so that its edge is a gap away
// from the wanted pairs. Interior windows, and blocks that leave too little
// room, use the solve's own (flat) filter polynomial.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "flz_internal.h"

namespace flz {

namespace {

double cheb_t(int d, double u) {
  if (std::fabs(u) <= 1.0) return std::cos(d * std::acos(u));
  const double v = std::cosh(d * std::acosh(std::fabs(u)));
  return (u < 0.0 && (d & 1)) ? -v : v;
}

}  // namespace

// Chebyshev coefficients (in z on [-1, 1]) of p(z) = T_d(a z + b) / T_d(-a + b),
// where z -> a z + b maps [zc, 1] onto [-1, 1]: at most 1 in magnitude on
// [-1, 1], 1 at z = -1, and at most 1 / |T_d(-a + b)| on [zc, 1]. By
// interpolation at the d + 1 Chebyshev points (exact for a degree-d
// polynomial up to rounding). Requires -1 < zc < 1.
void damping_coefficients(double zc, int d, double* out) {
  const double a = 2.0 / (1.0 - zc), b = -(1.0 + zc) / (1.0 - zc);
  const double norm = cheb_t(d, -a + b);
  std::vector<double> f(d + 1);
  for (int j = 0; j <= d; ++j) f[j] = cheb_t(d, a * std::cos(M_PI * (j + 0.5) / (d + 1)) + b) / norm;
  for (int k = 0; k <= d; ++k) {
    double s = 0.0;
    for (int j = 0; j <= d; ++j) s += f[j] * std::cos(M_PI * k * (j + 0.5) / (d + 1));
    out[k] = (k == 0 ? 1.0 : 2.0) * s / (d + 1);
  }
}

namespace {

using Clock = std::chrono::steady_clock;

// Rayleigh quotients and residual norms of the columns of X (n x kp, blocks of
// 16 columns, row-major) with AX = A X: out mu[j], res[j] (||Ax - mu x|| / ||x||).
void rayleigh(const flz_matrix* A, const double* X, double* AX, int64_t n, int kp, DevBuf<double>& dev,
              DevBuf<double>& part, std::vector<double>& mu, std::vector<double>& res, cudaStream_t st) {
  mu.assign(kp, 0.0);
  res.assign(kp, 0.0);
  for (int b = 0; b < kp / 16; ++b) {
    const double* Xb = X + (size_t)b * n * 16;
    double* AXb = AX + (size_t)b * n * 16;
    spmm(A, Xb, AXb, 16, 16, st);
    column_sums(Xb, Xb, nullptr, n, 16, 16, 0, dev.p, part.p, st);
    column_sums(Xb, AXb, nullptr, n, 16, 16, 0, dev.p + 16, part.p, st);
    double h[48];
    FLZ_CUDA(cudaMemcpyAsync(h, dev.p, sizeof(double) * 32, cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    for (int t = 0; t < 16; ++t) h[32 + t] = h[t] > 0.0 ? h[16 + t] / h[t] : 0.0;
    FLZ_CUDA(cudaMemcpyAsync(dev.p + 32, h + 32, sizeof(double) * 16, cudaMemcpyHostToDevice, st));
    column_sums(Xb, AXb, dev.p + 32, n, 16, 16, 1, dev.p + 48, part.p, st);
    double r2[16];
    FLZ_CUDA(cudaMemcpyAsync(r2, dev.p + 48, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    for (int t = 0; t < 16; ++t) {
      mu[b * 16 + t] = h[32 + t];
      res[b * 16 + t] = std::sqrt(std::max(r2[t], 0.0) / std::max(h[t], 1e-300));
    }
  }
}

// distance of mu to [alpha, beta] (0 inside)
inline double outside_by(double mu, double alpha, double beta) {
  return mu < alpha ? alpha - mu : (mu > beta ? mu - beta : 0.0);
}

}  // namespace

RefineResult refine(flz_matrix* A, const RefineArgs& g, double* X, int kp, cudaStream_t st, RefineWorkspace* ws) {
  const auto t0 = Clock::now();
  const int64_t n = A->n;
  RefineResult out;
  RefineWorkspace local;
  RefineWorkspace& w = ws ? *ws : local;
  DevBuf<double>&Y = w.Y, &AY = w.AY, &Vd = w.Vd, &dev = w.dev, &part = w.part, &S4 = w.S4, &T4 = w.T4;
  S4.reserve((size_t)n * 4);
  T4.reserve((size_t)n * 4);
  Y.reserve((size_t)n * kp);
  AY.reserve((size_t)n * kp);
  dev.reserve(64);
  part.reserve(column_sums_scratch(n, 16) + 64);
  const double c = 0.5 * (g.lmin + g.lmax), e = 0.5 * (g.lmax - g.lmin);
  const double anorm = std::max(std::fabs(g.lmin), std::fabs(g.lmax));
  const bool lower = g.alpha <= g.lmin, upper = g.beta >= g.lmax;
  std::vector<double> mu, res;
  rayleigh(A, X, AY.p, n, kp, dev, part, mu, res, st);
  double prev_worst = 1e300;
  for (int sweep = 0; sweep < g.max_sweeps; ++sweep) {
    // ---- the filter of this sweep ----
    // worst: the largest residual among the `wanted` best pairs in the window
    // (the block's extra columns may be poor approximations whose Rayleigh
    // quotients also fall in the window)
    std::vector<double> inres;
    double lo_blk = 1e300, hi_blk = -1e300;
    for (int j = 0; j < kp; ++j) {
      if (mu[j] >= g.alpha && mu[j] <= g.beta) inres.push_back(res[j] / anorm);
      lo_blk = std::min(lo_blk, mu[j]);
      hi_blk = std::max(hi_blk, mu[j]);
    }
    std::sort(inres.begin(), inres.end());
    const double worst =
        inres.empty() ? 1.0 : inres[std::min<size_t>(inres.size(), (size_t)std::max(g.wanted, 1)) - 1];
    // A start block that converges too slowly (judged from the second sweep
    // on) is given up: a sweep must halve the worst residual, and the
    // products still needed must fit the budget. At an end of the spectrum
    // the estimate is optimistic: the damping polynomial's asymptotic rate at
    // the window's edge, acosh|a z_w + b| per degree, with the damping
    // starting at the block's outermost Ritz value; for interior windows the
    // last sweep's rate is extrapolated.
    if (g.stop_on_stall && sweep >= 2) {
      const double rho = worst / prev_worst;
      if (!(rho <= 0.5)) break;
      if (g.matvec_budget > 0 && worst > g.tol) {
        double more_degrees;
        if (lower != upper) {
          const double edge = lower ? hi_blk : lo_blk;
          const double zc = std::min(lower ? (edge - c) / e : -(edge - c) / e, 1.0 - 1e-12);
          const double zw = lower ? (g.beta - c) / e : -(g.alpha - c) / e;
          const double u = std::fabs((2.0 * zw - (1.0 + zc)) / (1.0 - zc));
          more_degrees = u > 1.0 ? std::log(worst / g.tol) / std::acosh(u) : 1e300;
        } else {
          more_degrees = std::log(worst / g.tol) / std::log(1.0 / rho) * out.degrees.back();
        }
        if ((double)out.matvecs + more_degrees * kp > (double)g.matvec_budget) break;
      }
    }
    prev_worst = worst;
    std::vector<double> coeffs;
    // A polynomial with a large ratio between its values at the window's two
    // ends amplifies the errors of the pairs at the far end (about `worst` in
    // size) relative to those pairs themselves: keep that ratio below
    // 0.01 / worst, and use the flat solve filter where that leaves less than
    // a factor 20 of damping beyond the block.
    const double range_max = std::min(1e6, std::max(10.0, g.range_scale / std::max(worst, 1e-300)));
    const bool damp_ok = !(g.flat_first && sweep == 0);  // random extra columns: the window filter first
    if (damp_ok && ((lower && !upper && hi_blk > g.beta) || (upper && !lower && lo_blk < g.alpha))) {
      const double edge = lower ? hi_blk : lo_blk;
      const double zc = std::min(lower ? (edge - c) / e : -(edge - c) / e, 1.0 - 1e-12);  // damping interval [zc, 1]
      const double zw = lower ? (g.beta - c) / e : -(g.alpha - c) / e;   // the wanted end nearest it
      const double a = 2.0 / (1.0 - zc), b = -(1.0 + zc) / (1.0 - zc);
      const double uw = std::fabs(a * zw + b), u0 = std::fabs(b - a);     // at the near and far window ends
      // the least degree damping the interval by 10 worst / tol relative to
      // the window's near end, within the ratio bound across the window
      const double need = std::max(20.0, 10.0 * worst / g.tol);
      int d = 0;
      if (uw > 1.0)
        for (int t = 4; t <= g.max_degree; ++t) {
          if (t * (std::acosh(u0) - std::acosh(uw)) > std::log(range_max)) break;  // cosh ratio ~ exp of the difference
          d = t;
          if (std::cosh(t * std::acosh(uw)) >= need) break;
        }
      if (d >= 4 && std::cosh(d * std::acosh(uw)) >= 20.0) {
        coeffs.assign(d + 1, 0.0);
        damping_coefficients(zc, d, coeffs.data());
        if (upper)
          for (int k = 1; k <= d; k += 2) coeffs[k] = -coeffs[k];  // p(z) = q(-z)
      }
    }
    // interior window, or too little room: the solve's own (flat) filter, at
    // half its degree in the first sweep (FP32 errors need a factor of tens)
    if (coeffs.empty()) coeffs = (sweep == 0 && g.filter_half.size() > 1) ? g.filter_half : g.filter;
    out.degrees.push_back((int)coeffs.size() - 1);
    const int m = (int)coeffs.size() - 1;
    out.matvecs += (int64_t)kp * m;
    // the filter runs on 4-column slices of the 16-column blocks (its fastest width)
    const bool extras_only = g.flat_first && sweep == 0;
    if (extras_only) out.matvecs -= (int64_t)(g.wanted / 4 * 4) * m;
    for (int b = 0; b < kp / 16; ++b)
      for (int q = 0; q < 4; ++q) {
        if (extras_only && 16 * b + 4 * q + 4 <= g.wanted) {  // a slice of start vectors: Y = X
          FLZ_CUDA(cudaMemcpy2DAsync(Y.p + (size_t)b * n * 16 + 4 * q, 16 * sizeof(double),
                                     X + (size_t)b * n * 16 + 4 * q, 16 * sizeof(double), 4 * sizeof(double),
                                     (size_t)n, cudaMemcpyDeviceToDevice, st));
          continue;
        }
        FLZ_CUDA(cudaMemcpy2DAsync(S4.p, 4 * sizeof(double), X + (size_t)b * n * 16 + 4 * q, 16 * sizeof(double),
                                   4 * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice, st));
        filter_apply(A, c, e, coeffs.data(), m, 4, S4.p, T4.p, FLZ_PREC_FX64, FLZ_REC_FORWARD, st);
        FLZ_CUDA(cudaMemcpy2DAsync(Y.p + (size_t)b * n * 16 + 4 * q, 16 * sizeof(double), T4.p, 4 * sizeof(double),
                                   4 * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice, st));
      }
    out.filter_precision = A->last_filter_precision;
    // ---- Rayleigh-Ritz on A in the span of Y ----
    TcBasis& tb = w.tb;
    tb.reshape(n, kp, st);
    for (int b = 0; b < kp / 16; ++b) tb.append(Y.p + (size_t)b * n * 16, 16, 16 * b, st);  // rounds Y to the grid
    Vd.reserve((size_t)kp * kp);
    DevBuf<double>&Md = w.Md, &Hd = w.Hd;
    Md.reserve((size_t)kp * kp);
    Hd.reserve((size_t)kp * kp);
    for (int b = 0; b < kp / 16; ++b) {
      const double* Yb = Y.p + (size_t)b * n * 16;
      double* AYb = AY.p + (size_t)b * n * 16;
      spmm(A, Yb, AYb, 16, 16, st);
      tb.column_max(Yb, 16, 16, tb.wmax.p, st);
      tb.project(kp, Yb, 16, 16, tb.wmax.p, Md.p + 16 * b, kp, st);
      tb.column_max(AYb, 16, 16, tb.wmax.p, st);
      tb.project(kp, AYb, 16, 16, tb.wmax.p, Hd.p + 16 * b, kp, st);
    }
    std::vector<double> M((size_t)kp * kp), H((size_t)kp * kp);
    FLZ_CUDA(cudaMemcpyAsync(M.data(), Md.p, sizeof(double) * kp * kp, cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaMemcpyAsync(H.data(), Hd.p, sizeof(double) * kp * kp, cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaMemcpyAsync(tb.status_host, tb.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    tb.check_status();
    for (int i = 0; i < kp; ++i)
      for (int j = 0; j < i; ++j) {
        M[(size_t)i * kp + j] = M[(size_t)j * kp + i] = 0.5 * (M[(size_t)i * kp + j] + M[(size_t)j * kp + i]);
        H[(size_t)i * kp + j] = H[(size_t)j * kp + i] = 0.5 * (H[(size_t)i * kp + j] + H[(size_t)j * kp + i]);
      }
    // D M D = U S U^T with D = diag(M)^(-1/2) (unit columns); Z = D U_kept S^(-1/2)
    // over the numerically independent directions
    std::vector<double> dsc(kp);
    for (int i = 0; i < kp; ++i) dsc[i] = 1.0 / std::sqrt(std::max(M[(size_t)i * kp + i], 1e-300));
    std::vector<double> sw, U;
    std::vector<double> Mc((size_t)kp * kp);
    for (int i = 0; i < kp; ++i)
      for (int j = 0; j < kp; ++j) Mc[(size_t)i * kp + j] = dsc[i] * M[(size_t)i * kp + j] * dsc[j];
    dense_sym_eig(Mc, kp, sw, U);
    const double smax = std::max(sw.back(), 1e-300);
    std::vector<int> keep;
    for (int i = 0; i < kp; ++i)
      if (sw[i] > 1e-12 * smax) keep.push_back(i);
    const int ke = (int)keep.size();
    std::vector<double> Z((size_t)kp * ke);
    for (int i = 0; i < kp; ++i)
      for (int q = 0; q < ke; ++q) Z[(size_t)i * ke + q] = dsc[i] * U[(size_t)i * kp + keep[q]] / std::sqrt(sw[keep[q]]);
    // C = Z^T H Z
    std::vector<double> HZ((size_t)kp * ke, 0.0), Cm((size_t)ke * ke, 0.0);
    for (int i = 0; i < kp; ++i)
      for (int l = 0; l < kp; ++l) {
        const double h = H[(size_t)i * kp + l];
        if (h == 0.0) continue;
        const double* zr = &Z[(size_t)l * ke];
        double* out_r = &HZ[(size_t)i * ke];
        for (int q = 0; q < ke; ++q) out_r[q] += h * zr[q];
      }
    for (int l = 0; l < kp; ++l) {
      const double* zr = &Z[(size_t)l * ke];
      const double* hz = &HZ[(size_t)l * ke];
      for (int p_ = 0; p_ < ke; ++p_) {
        const double zv = zr[p_];
        double* cr = &Cm[(size_t)p_ * ke];
        for (int q = 0; q < ke; ++q) cr[q] += zv * hz[q];
      }
    }
    std::vector<double> theta, Wv;
    dense_sym_eig(Cm, ke, theta, Wv);
    // keep the pairs nearest the window, as many as fill whole blocks of 16
    std::vector<int> ord(ke);
    for (int i = 0; i < ke; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      return outside_by(theta[x], g.alpha, g.beta) < outside_by(theta[y], g.alpha, g.beta);
    });
    const int kn = std::max(16, (std::min(ke, kp) / 16) * 16);
    if (ke < kn) fail(FLZ_ERR_NOT_CONVERGED, "refinement: the filtered block lost its rank (%d of %d)", ke, kp);
    // V = Z W restricted to the kept pairs (kp x kn, row-major)
    std::vector<double> V((size_t)kp * kn, 0.0);
    for (int i = 0; i < kp; ++i)
      for (int q = 0; q < kn; ++q) {
        const int col = ord[q];
        double v = 0.0;
        for (int p_ = 0; p_ < ke; ++p_) v += Z[(size_t)i * ke + p_] * Wv[(size_t)p_ * ke + col];
        V[(size_t)i * kn + q] = v;
      }
    Vd.reserve((size_t)kp * kn);
    FLZ_CUDA(cudaMemcpyAsync(Vd.p, V.data(), sizeof(double) * kp * kn, cudaMemcpyHostToDevice, st));
    for (int b = 0; b < kn / 16; ++b) tb.multiply(kp, Vd.p + 16 * b, kn, 16, X + (size_t)b * n * 16, 16, st);
    FLZ_CUDA(cudaMemcpyAsync(tb.status_host, tb.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    tb.check_status();
    kp = kn;
    rayleigh(A, X, AY.p, n, kp, dev, part, mu, res, st);
    out.sweeps = sweep + 1;
    bool done = true;
    for (int j = 0; j < kp; ++j)
      if (mu[j] >= g.alpha && mu[j] <= g.beta && !(res[j] / anorm <= g.tol)) done = false;
    if (done) {
      out.converged = true;
      break;
    }
  }
  out.kp = kp;
  for (int j = 0; j < kp; ++j)
    if (mu[j] >= g.alpha && mu[j] <= g.beta) {
      out.index.push_back(j);
      out.vals.push_back(mu[j]);
      out.res.push_back(res[j] / anorm);
    } else {
      ++out.outside;
    }
  out.ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  return out;
}

}  // namespace flz
