// extern "C" entry points of include/flz.h. Each catches the internal
// flz::Failure so that no exception crosses the ABI.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "flz_internal.h"

namespace flz {

namespace {
thread_local std::string g_last_error;
}
thread_local int64_t g_kernel_launches = 0;
std::atomic<uint64_t> g_wait_ns{2000000000ull};
uint64_t wait_limit_ns() { return g_wait_ns.load(); }

void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
void clear_last_error() { g_last_error.clear(); }

[[noreturn]] void fail(flz_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  throw Failure{st};
}

// Section 2.2: b_0 = (acos a - acos b)/pi, b_i = 2 (sin(i acos a) - sin(i acos b)) / (i pi).
void chebyshev_coefficients(double a, double b, int m, double* out) {
  const double ta = std::acos(a), tb = std::acos(b);
  out[0] = (ta - tb) / M_PI;
  for (int i = 1; i <= m; ++i) out[i] = 2.0 * (std::sin(i * ta) - std::sin(i * tb)) / (i * M_PI);
}

namespace {
// integral of cos(k t) dt and of cos(t) cos(k t) dt (antiderivatives at t)
double int_cos(int k, double t) { return k == 0 ? t : std::sin(k * t) / k; }
double int_zcos(int k, double t) {
  if (k == 1) return 0.5 * (t + 0.5 * std::sin(2.0 * t));
  return 0.5 * (std::sin((k - 1) * t) / (k - 1) + std::sin((k + 1) * t) / (k + 1));
}
}  // namespace

// Weighted least-squares (truncated Chebyshev series) coefficients of the
// smoothed step: 1 on [a, b], linear ramps of width d down to 0 outside,
// clipped to [-1, 1]; piecewise closed forms in t = arccos z.
void smoothed_step_coefficients(double a, double b, double d, int m, double* out) {
  struct Piece {
    double z_lo, z_hi;
    bool ramp;
    double z0, z1;  // ramp value (z - z0) / (z1 - z0)
  };
  std::vector<Piece> pieces;
  const double flo = std::max(a, -1.0), fhi = std::min(b, 1.0);
  if (fhi > flo) pieces.push_back({flo, fhi, false, 0.0, 0.0});
  if (d > 0.0) {
    const double l0 = std::max(a - d, -1.0), l1 = std::min(a, 1.0);
    if (l1 > l0) pieces.push_back({l0, l1, true, a - d, a});
    const double r0 = std::max(b, -1.0), r1 = std::min(b + d, 1.0);
    if (r1 > r0) pieces.push_back({r0, r1, true, b + d, b});
  }
  for (int k = 0; k <= m; ++k) {
    double acc = 0.0;
    for (const Piece& pc : pieces) {
      const double t_lo = std::acos(pc.z_hi), t_hi = std::acos(pc.z_lo);
      const double ic = int_cos(k, t_hi) - int_cos(k, t_lo);
      if (!pc.ramp)
        acc += ic;
      else
        acc += ((int_zcos(k, t_hi) - int_zcos(k, t_lo)) - pc.z0 * ic) / (pc.z1 - pc.z0);
    }
    out[k] = (k == 0 ? 1.0 : 2.0) / M_PI * acc;
  }
}

void jackson_factors(int m, double* g) {
  const double a = M_PI / (m + 1);
  for (int k = 0; k <= m; ++k) g[k] = ((m - k + 1) * std::cos(k * a) + std::sin(k * a) / std::tan(a)) / (m + 1);
}

void lanczos_sigma_factors(int m, double* g) {
  g[0] = 1.0;
  for (int k = 1; k <= m; ++k) {
    const double x = k * M_PI / (m + 1);
    g[k] = std::sin(x) / x;
  }
}

void filter_coeffs_for(const flz_params& p, double a, double b, int m, double* out) {
  if (p.transition > 0.0)
    smoothed_step_coefficients(a, b, p.transition, m, out);
  else
    chebyshev_coefficients(a, b, m, out);
  if (p.damping != 0) {
    std::vector<double> g(m + 1);
    damping_factors(p.damping, m, g.data());
    for (int k = 0; k <= m; ++k) out[k] *= g[k];
  }
}

void damping_factors(int damping, int m, double* g) {
  if (damping == 1)
    jackson_factors(m, g);
  else if (damping == 2)
    lanczos_sigma_factors(m, g);
  else
    for (int k = 0; k <= m; ++k) g[k] = 1.0;
}

// Eq. (optimaldegree): least m with ||p_m - phi||^2 < eps^2 ||phi||^2 in the
// weighted Chebyshev norm, the error by Parseval: ||phi||^2 = acos a - acos b,
// ||p_m||^2 = pi b_0^2 + (pi/2) sum_{i=1..m} b_i^2. Returns -1 if none <= max_degree.
int auto_degree(double a, double b, double eps, int max_degree) {
  const double ta = std::acos(a), tb = std::acos(b);
  const double phi2 = ta - tb;
  const double b0 = phi2 / M_PI;
  double kept = M_PI * b0 * b0;
  for (int m = 1; m <= max_degree; ++m) {
    const double bm = 2.0 * (std::sin(m * ta) - std::sin(m * tb)) / (m * M_PI);
    kept += 0.5 * M_PI * bm * bm;
    if (phi2 - kept < eps * eps * phi2) return m;
  }
  return -1;
}

flz_status solve(flz_solver* s, cudaStream_t st);
flz_status solve_sliced(flz_solver* s, int nslices, cudaStream_t st);
void bounds_entry(flz_matrix* A, int steps, int r, uint64_t seed, cudaStream_t st, double* lmin, double* lmax);

}  // namespace flz


using flz::fail;

namespace {

// The filter folds the shift -cI into the stored diagonal, so every row must
// store a_ii; rows that do not get an explicit zero (same matrix).
void insert_zero_diagonals(flz_matrix* A) {
  const int64_t n = A->n, nnz = A->nnz;
  std::vector<int32_t> rp(n + 1), cl(nnz), rp2(n + 1), cl2;
  std::vector<double> vl(nnz), vl2;
  FLZ_CUDA(cudaMemcpy(rp.data(), A->rowptr.p, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
  if (nnz > 0) {
    FLZ_CUDA(cudaMemcpy(cl.data(), A->col.p, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
    FLZ_CUDA(cudaMemcpy(vl.data(), A->val.p, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
  }
  cl2.reserve(nnz + n);
  vl2.reserve(nnz + n);
  rp2[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    bool done = false;
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j) {
      if (!done && cl[j] >= i) {
        if (cl[j] != i) {
          cl2.push_back((int32_t)i);
          vl2.push_back(0.0);
        }
        done = true;
      }
      cl2.push_back(cl[j]);
      vl2.push_back(vl[j]);
    }
    if (!done) {
      cl2.push_back((int32_t)i);
      vl2.push_back(0.0);
    }
    if ((int64_t)cl2.size() > 2147483647LL) fail(FLZ_ERR_INVALID_ARG, "nnz with diagonals exceeds int32");
    rp2[i + 1] = (int32_t)cl2.size();
  }
  A->nnz = (int64_t)cl2.size();
  A->col.reserve((size_t)A->nnz);
  A->val.reserve((size_t)A->nnz);
  FLZ_CUDA(cudaMemcpy(A->rowptr.p, rp2.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
  FLZ_CUDA(cudaMemcpy(A->col.p, cl2.data(), sizeof(int32_t) * A->nnz, cudaMemcpyHostToDevice));
  FLZ_CUDA(cudaMemcpy(A->val.p, vl2.data(), sizeof(double) * A->nnz, cudaMemcpyHostToDevice));
  if (flz::find_diagonals(A) != 0) fail(FLZ_ERR_BAD_CSR, "diagonal insertion failed");
}

}  // namespace

extern "C" {

const char* flz_status_string(flz_status s) {
  switch (s) {
    case FLZ_OK: return "FLZ_OK";
    case FLZ_ERR_INVALID_ARG: return "FLZ_ERR_INVALID_ARG";
    case FLZ_ERR_NOT_SYMMETRIC: return "FLZ_ERR_NOT_SYMMETRIC";
    case FLZ_ERR_BAD_CSR: return "FLZ_ERR_BAD_CSR";
    case FLZ_ERR_EMPTY_INTERVAL: return "FLZ_ERR_EMPTY_INTERVAL";
    case FLZ_ERR_NOT_CONVERGED: return "FLZ_ERR_NOT_CONVERGED";
    case FLZ_ERR_OUT_OF_MEMORY: return "FLZ_ERR_OUT_OF_MEMORY";
    case FLZ_ERR_CUDA: return "FLZ_ERR_CUDA";
    case FLZ_ERR_TIMEOUT: return "FLZ_ERR_TIMEOUT";
    case FLZ_ERR_CAPACITY: return "FLZ_ERR_CAPACITY";
    case FLZ_ERR_NO_INTERVAL: return "FLZ_ERR_NO_INTERVAL";
    case FLZ_ERR_NOT_SOLVED: return "FLZ_ERR_NOT_SOLVED";
  }
  return "FLZ_ERR_UNKNOWN";
}

const char* flz_last_error(void) { return flz::g_last_error.c_str(); }

flz_status flz_params_default(flz_params* p) {
  if (!p) return FLZ_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->block_size = 3;
  p->degree = 0;
  p->degree_eps = 0.3123;
  p->max_degree = 2000;
  p->tol = 1e-10;
  p->check_every = 30;
  p->max_basis = 0;
  p->guard = 0;
  p->precision = FLZ_PREC_FP64;
  p->bounds_steps = 60;
  p->seed = 1;
  p->lmin = 0.0;
  p->lmax = 0.0;
  p->damping = 0;
  p->recurrence = FLZ_REC_FORWARD;
  p->transition = 0.0;
  p->ortho = FLZ_ORTHO_AUTO;
  p->start_mode = FLZ_START_KRYLOV;
  return FLZ_OK;
}

flz_status flz_filter_coefficients(double alpha, double beta, int32_t degree, double* out) {
  FLZ_API_BEGIN
  if (!out || degree < 0) fail(FLZ_ERR_INVALID_ARG, "out is NULL or degree < 0");
  if (!(alpha >= -1.0 && beta <= 1.0 && alpha < beta)) fail(FLZ_ERR_INVALID_ARG, "need -1 <= alpha < beta <= 1");
  flz::chebyshev_coefficients(alpha, beta, degree, out);
  FLZ_API_END
}

flz_status flz_smoothed_step_coefficients(double alpha, double beta, double delta, int32_t degree, double* out) {
  FLZ_API_BEGIN
  if (!out || degree < 0) fail(FLZ_ERR_INVALID_ARG, "out is NULL or degree < 0");
  if (!(alpha >= -1.0 && beta <= 1.0 && alpha < beta && delta >= 0.0))
    fail(FLZ_ERR_INVALID_ARG, "need -1 <= alpha < beta <= 1 and delta >= 0");
  flz::smoothed_step_coefficients(alpha, beta, delta, degree, out);
  FLZ_API_END
}

flz_status flz_jackson_factors(int32_t degree, double* out) {
  FLZ_API_BEGIN
  if (!out || degree < 0) fail(FLZ_ERR_INVALID_ARG, "out is NULL or degree < 0");
  flz::jackson_factors(degree, out);
  FLZ_API_END
}

flz_status flz_lanczos_sigma_factors(int32_t degree, double* out) {
  FLZ_API_BEGIN
  if (!out || degree < 0) fail(FLZ_ERR_INVALID_ARG, "out is NULL or degree < 0");
  flz::lanczos_sigma_factors(degree, out);
  FLZ_API_END
}

flz_status flz_damping_coefficients(double zc, int32_t degree, double* out) {
  FLZ_API_BEGIN
  if (!out || degree < 0 || !(zc > -1.0 && zc < 1.0)) fail(FLZ_ERR_INVALID_ARG, "need -1 < zc < 1, degree >= 0");
  flz::damping_coefficients(zc, degree, out);
  FLZ_API_END
}

flz_status flz_filter_degree(double alpha, double beta, double eps, int32_t max_degree, int32_t* degree) {
  FLZ_API_BEGIN
  if (!degree || max_degree < 1 || !(eps > 0.0)) fail(FLZ_ERR_INVALID_ARG, "bad degree arguments");
  if (!(alpha >= -1.0 && beta <= 1.0 && alpha < beta)) fail(FLZ_ERR_INVALID_ARG, "need -1 <= alpha < beta <= 1");
  const int m = flz::auto_degree(alpha, beta, eps, max_degree);
  if (m < 0) fail(FLZ_ERR_CAPACITY, "no degree <= %d satisfies the rule", max_degree);
  *degree = m;
  FLZ_API_END
}

flz_status flz_matrix_create_csr(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                                 const void* val, flz_dtype val_type, flz_memspace where, int32_t check_symmetry,
                                 flz_matrix** out) {
  FLZ_API_BEGIN
  if (!out) fail(FLZ_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || nnz < 0 || n > 2147483647LL || nnz > 2147483647LL) fail(FLZ_ERR_INVALID_ARG, "n/nnz out of range");
  if (!rowptr || (nnz > 0 && (!col || !val))) fail(FLZ_ERR_INVALID_ARG, "null CSR array");
  if (val_type != FLZ_F64 && val_type != FLZ_F32) fail(FLZ_ERR_INVALID_ARG, "values must be FLZ_F64 or FLZ_F32");
  if (where != FLZ_HOST && where != FLZ_DEVICE) fail(FLZ_ERR_INVALID_ARG, "bad memspace");
  flz_matrix* A = new flz_matrix();
  try {
    A->n = n;
    A->nnz = nnz;
    FLZ_CUDA(cudaGetDevice(&A->device));
    A->rowptr.reserve((size_t)n + 1);
    A->col.reserve((size_t)std::max<int64_t>(nnz, 1));
    A->val.reserve((size_t)std::max<int64_t>(nnz, 1));
    const cudaMemcpyKind kind = where == FLZ_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    FLZ_CUDA(cudaMemcpy(A->rowptr.p, rowptr, sizeof(int32_t) * (n + 1), kind));
    if (nnz > 0) {
      FLZ_CUDA(cudaMemcpy(A->col.p, col, sizeof(int32_t) * nnz, kind));
      if (val_type == FLZ_F64) {
        FLZ_CUDA(cudaMemcpy(A->val.p, val, sizeof(double) * nnz, kind));
      } else {
        std::vector<float> hf;
        const float* src = static_cast<const float*>(val);
        if (where == FLZ_DEVICE) {
          hf.resize(nnz);
          FLZ_CUDA(cudaMemcpy(hf.data(), val, sizeof(float) * nnz, cudaMemcpyDeviceToHost));
          src = hf.data();
        }
        std::vector<double> hd(src, src + nnz);
        FLZ_CUDA(cudaMemcpy(A->val.p, hd.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice));
      }
    }
    const flz_status vs = flz::validate_csr(A, check_symmetry);
    if (vs == FLZ_ERR_BAD_CSR) fail(vs, "CSR structure invalid (rowptr, column range or column order)");
    if (vs == FLZ_ERR_NOT_SYMMETRIC) fail(vs, "matrix is not symmetric");
    A->nnz_user = nnz;
    if (flz::find_diagonals(A) > 0) insert_zero_diagonals(A);
    flz::gershgorin(A, &A->glo, &A->ghi, &A->max_row_nnz);
    A->max_cta_nnz = flz::max_block_nnz(A, 256);
    flz::build_sell(A);
    if (A->max_row_nnz > flz::kLongRow) {
      std::vector<int32_t> rp(A->n + 1), lr;
      FLZ_CUDA(cudaMemcpy(rp.data(), A->rowptr.p, sizeof(int32_t) * (A->n + 1), cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < A->n; ++i)
        if (rp[i + 1] - rp[i] > flz::kLongRow) lr.push_back((int32_t)i);
      A->n_long = (int32_t)lr.size();
      A->long_rows.reserve(lr.size());
      FLZ_CUDA(cudaMemcpy(A->long_rows.p, lr.data(), sizeof(int32_t) * lr.size(), cudaMemcpyHostToDevice));
    }
  } catch (...) {
    delete A;
    throw;
  }
  *out = A;
  FLZ_API_END
}

flz_status flz_matrix_destroy(flz_matrix* A) {
  FLZ_API_BEGIN
  delete A;
  FLZ_API_END
}

flz_status flz_matrix_info(const flz_matrix* A, int64_t* n, int64_t* nnz, double* glo, double* ghi) {
  FLZ_API_BEGIN
  if (!A) fail(FLZ_ERR_INVALID_ARG, "matrix is NULL");
  if (n) *n = A->n;
  if (nnz) *nnz = A->nnz_user;
  if (glo) *glo = A->glo;
  if (ghi) *ghi = A->ghi;
  FLZ_API_END
}

flz_status flz_matrix_format(const flz_matrix* A, int32_t* sell, int64_t* sell_entries, int32_t* long_rows) {
  FLZ_API_BEGIN
  if (!A) fail(FLZ_ERR_INVALID_ARG, "matrix is NULL");
  if (sell) *sell = A->sell ? 1 : 0;
  if (sell_entries) *sell_entries = A->sell ? A->sell_len : 0;
  if (long_rows) *long_rows = A->n_long;
  FLZ_API_END
}

flz_status flz_filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int32_t degree, int32_t r,
                            const double* V, double* W, int32_t precision, int32_t recurrence, void* stream) {
  FLZ_API_BEGIN
  if (!A || !coeffs || !V || !W) fail(FLZ_ERR_INVALID_ARG, "null argument");
  if (recurrence != FLZ_REC_FORWARD && recurrence != FLZ_REC_CLENSHAW) fail(FLZ_ERR_INVALID_ARG, "bad recurrence");
  if (degree < 0 || r < 1 || r > 16 || !(e > 0.0)) fail(FLZ_ERR_INVALID_ARG, "need degree >= 0, 1 <= r <= 16, e > 0");
  if (precision < FLZ_PREC_FP64 || precision > FLZ_PREC_FX64) fail(FLZ_ERR_INVALID_ARG, "bad precision");
  const size_t bytes = sizeof(double) * (size_t)A->n * r;
  const char* v = reinterpret_cast<const char*>(V);
  const char* w = reinterpret_cast<const char*>(W);
  if (v < w + bytes && w < v + bytes) fail(FLZ_ERR_INVALID_ARG, "V and W overlap");
  flz::filter_apply(A, c, e, coeffs, degree, r, V, W, precision, recurrence, static_cast<cudaStream_t>(stream));
  if (precision == FLZ_PREC_FX64) {  // a range overflow is reported here, not by a later call
    FLZ_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    flz::fx_check_flag(A);
  }
  FLZ_API_END
}

flz_status flz_spectrum_bounds(flz_matrix* A, int32_t steps, int32_t r, uint64_t seed, double* lmin, double* lmax,
                               void* stream) {
  FLZ_API_BEGIN
  if (!A || !lmin || !lmax) fail(FLZ_ERR_INVALID_ARG, "null argument");
  if (steps < 1 || r < 1 || r > 16 || r > A->n) fail(FLZ_ERR_INVALID_ARG, "bad steps or block width");
  flz::bounds_entry(A, steps, r, seed, static_cast<cudaStream_t>(stream), lmin, lmax);
  FLZ_API_END
}

flz_status flz_band_eigenvalues(int32_t K, int32_t b, const double* T, double* theta) {
  FLZ_API_BEGIN
  if (K < 1 || b < 0 || !T || !theta) fail(FLZ_ERR_INVALID_ARG, "bad band matrix arguments");
  std::vector<double> t(T, T + (size_t)K * K), th;
  flz::band_eigenvalues(t, K, std::min<int32_t>(std::max<int32_t>(b, 1), K), th);
  for (int i = 0; i < K; ++i) theta[i] = th[i];
  FLZ_API_END
}

flz_status flz_band_eigenvectors(int32_t K, int32_t b, const double* T, const double* theta, int32_t count,
                                 const int32_t* idx, double* Y, uint64_t seed) {
  FLZ_API_BEGIN
  if (K < 1 || b < 0 || !T || !theta || count < 0 || (count > 0 && (!idx || !Y)))
    fail(FLZ_ERR_INVALID_ARG, "bad band matrix arguments");
  std::vector<double> t(T, T + (size_t)K * K), th(theta, theta + K), y;
  std::vector<int> ix(idx, idx + count);
  for (int v : ix)
    if (v < 0 || v >= K) fail(FLZ_ERR_INVALID_ARG, "eigenvalue index out of range");
  flz::band_eigenvectors(t, K, std::min<int32_t>(std::max<int32_t>(b, 1), K), th, ix, y, seed);
  for (size_t i = 0; i < y.size(); ++i) Y[i] = y[i];
  FLZ_API_END
}

flz_status flz_sym_eig(int32_t n, const double* S, double* w, double* Z) {
  FLZ_API_BEGIN
  if (n < 1 || !S || !w || !Z) fail(FLZ_ERR_INVALID_ARG, "bad arguments");
  std::vector<double> A(S, S + (size_t)n * n), ww, zz;
  flz::dense_sym_eig(A, n, ww, zz);
  std::copy(ww.begin(), ww.end(), w);
  std::copy(zz.begin(), zz.end(), Z);
  FLZ_API_END
}

namespace {

void check_basis_args(int64_t n, int32_t nb, int32_t r, const double* Q, const double* W, const double* C,
                      int32_t method) {
  if (n < 1 || nb < 1 || r < 1 || r > 16 || !Q || !W || !C) fail(FLZ_ERR_INVALID_ARG, "bad arguments");
  if (method != FLZ_ORTHO_CUDA_CORES && method != FLZ_ORTHO_TENSOR) fail(FLZ_ERR_INVALID_ARG, "bad method");
  if (method == FLZ_ORTHO_TENSOR && !flz::TcBasis::supported(r))
    fail(FLZ_ERR_INVALID_ARG, "the tensor-core path takes block widths 1..16");
}

// Digit copy of a caller's basis (the caller's FP64 values stay untouched).
void digits_of(flz::TcBasis& B, int64_t n, int32_t nb, int32_t r, const double* Q, cudaStream_t st) {
  B.reserve(n, (int64_t)nb * r);
  flz::DevBuf<double> tmp;
  tmp.reserve((size_t)n * r);
  for (int b = 0; b < nb; ++b) {
    FLZ_CUDA(cudaMemcpyAsync(tmp.p, Q + (size_t)b * n * r, sizeof(double) * n * r, cudaMemcpyDeviceToDevice, st));
    B.append(tmp.p, r, b * r, st);
  }
  FLZ_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

flz_status flz_basis_project(int64_t n, int32_t nb, int32_t r, const double* Q, const double* W, double* C,
                             int32_t method, void* stream) {
  FLZ_API_BEGIN
  check_basis_args(n, nb, r, Q, W, C, method);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (method == FLZ_ORTHO_CUDA_CORES) {
    flz::DevBuf<double> part;
    part.reserve(std::max(flz::basis_dot_scratch(n, nb, r, r), (size_t)1));
    flz::basis_dot(Q, nb, n, r, W, r, r, C, part.p, st);
    FLZ_CUDA(cudaStreamSynchronize(st));
  } else {
    flz::TcBasis B;
    digits_of(B, n, nb, r, Q, st);
    B.column_max(W, r, r, B.wmax.p, st);
    B.project(nb * r, W, r, r, B.wmax.p, C, r, st);
    FLZ_CUDA(cudaMemcpyAsync(B.status_host, B.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    B.check_status();
  }
  FLZ_API_END
}

flz_status flz_basis_orthogonalize(int64_t n, int32_t nb, int32_t r, const double* Q, double* W, double* C,
                                   int32_t method, void* stream) {
  FLZ_API_BEGIN
  check_basis_args(n, nb, r, Q, W, C, method);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t kr = (size_t)nb * r * r;
  flz::DevBuf<double> C2;
  C2.reserve(kr);
  if (method == FLZ_ORTHO_CUDA_CORES) {
    flz::DevBuf<double> part;
    part.reserve(std::max(flz::basis_dot_scratch(n, nb, r, r), (size_t)1));
    flz::basis_dot(Q, nb, n, r, W, r, r, C, part.p, st);
    flz::basis_update(Q, nb, n, r, C, r, -1.0, 1.0, W, r, st);
    flz::basis_dot(Q, nb, n, r, W, r, r, C2.p, part.p, st);
    flz::basis_update(Q, nb, n, r, C2.p, r, -1.0, 1.0, W, r, st);
    FLZ_CUDA(cudaStreamSynchronize(st));
  } else {
    flz::TcBasis B;
    digits_of(B, n, nb, r, Q, st);
    B.cgs2(nb * r, W, r, C, C2.p, st);
    FLZ_CUDA(cudaStreamSynchronize(st));
    B.check_status();
  }
  std::vector<double> c1(kr), c2(kr);
  FLZ_CUDA(cudaMemcpy(c1.data(), C, sizeof(double) * kr, cudaMemcpyDeviceToHost));
  FLZ_CUDA(cudaMemcpy(c2.data(), C2.p, sizeof(double) * kr, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < kr; ++i) c1[i] += c2[i];
  FLZ_CUDA(cudaMemcpy(C, c1.data(), sizeof(double) * kr, cudaMemcpyHostToDevice));
  FLZ_API_END
}

flz_status flz_basis_multiply(int64_t n, int32_t nb, int32_t r, const double* Q, const double* H, int32_t s,
                              double* X, int32_t method, void* stream) {
  FLZ_API_BEGIN
  check_basis_args(n, nb, r, Q, H, X, method);
  if (s < 1 || s > 16) fail(FLZ_ERR_INVALID_ARG, "s must be in 1..16");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (method == FLZ_ORTHO_CUDA_CORES) {
    flz::basis_update(Q, nb, n, r, H, s, 1.0, 0.0, X, s, st);
    FLZ_CUDA(cudaStreamSynchronize(st));
  } else {
    flz::TcBasis B;
    digits_of(B, n, nb, r, Q, st);
    B.multiply(nb * r, H, s, s, X, s, st);
    FLZ_CUDA(cudaMemcpyAsync(B.status_host, B.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FLZ_CUDA(cudaStreamSynchronize(st));
    B.check_status();
  }
  FLZ_API_END
}

flz_status flz_measure_alu_peak(int32_t kind, double* ops_per_s) {
  FLZ_API_BEGIN
  if (!ops_per_s || (kind != 0 && kind != 1)) fail(FLZ_ERR_INVALID_ARG, "kind must be 0 (FP64 FMA) or 1 (integer)");
  *ops_per_s = flz::measure_alu_peak(kind);
  FLZ_API_END
}

flz_status flz_set_wait_limit(uint64_t ns, uint64_t* previous) {
  FLZ_API_BEGIN
  const uint64_t old = flz::g_wait_ns.exchange(ns);
  if (previous) *previous = old;
  FLZ_API_END
}

flz_status flz_tc_mma_probe(const uint16_t* a_img, int64_t a_bytes, const uint16_t* b_img, int64_t b_bytes,
                            int32_t n, int32_t a_mn_major, int32_t a_lbo, int32_t a_sbo, int32_t b_lbo,
                            int32_t b_sbo, float* d) {
  FLZ_API_BEGIN
  if (!a_img || !b_img || !d || a_bytes < 16 || b_bytes < 16 || a_lbo < 0 || a_sbo < 0 || b_lbo < 0 || b_sbo < 0 ||
      (a_mn_major != 0 && a_mn_major != 1))
    fail(FLZ_ERR_INVALID_ARG, "bad arguments");
  const int st = flz::tc_probe(a_img, (size_t)a_bytes, b_img, (size_t)b_bytes, n, a_mn_major, (uint32_t)a_lbo,
                               (uint32_t)a_sbo, (uint32_t)b_lbo, (uint32_t)b_sbo, d);
  if (st) fail(FLZ_ERR_TIMEOUT, "the MMA's completion wait expired");
  FLZ_API_END
}

flz_status flz_solver_create(flz_matrix* A, const flz_params* params, flz_solver** out) {
  FLZ_API_BEGIN
  if (!A || !out) fail(FLZ_ERR_INVALID_ARG, "null argument");
  flz_params p;
  if (params) p = *params;
  else flz_params_default(&p);
  if (p.block_size < 1 || p.block_size > 16 || p.block_size > A->n) fail(FLZ_ERR_INVALID_ARG, "block_size must be in [1, min(16, n)]");
  if (p.degree < 0 || p.max_degree < 1 || p.check_every < 1 || !(p.tol > 0.0) || !(p.degree_eps > 0.0) ||
      p.bounds_steps < 1 || p.max_basis < 0 || p.guard < 0 || p.damping < 0 || p.damping > 2 || !(p.transition >= 0.0) ||
      (p.recurrence != FLZ_REC_FORWARD && p.recurrence != FLZ_REC_CLENSHAW) || p.ortho < FLZ_ORTHO_AUTO ||
      p.ortho > FLZ_ORTHO_TENSOR || p.refine < 0 || p.refine > 1 ||
      (p.start_mode != FLZ_START_KRYLOV && p.start_mode != FLZ_START_SUBSPACE) || p.persistent < 0 ||
      p.persistent > 1 || (p.tile_rows != 0 && p.tile_rows != 128 && p.tile_rows != 256))
    fail(FLZ_ERR_INVALID_ARG, "invalid parameter");
  if (p.ortho == FLZ_ORTHO_TENSOR && (!flz::TcBasis::supported(p.block_size) || p.precision == FLZ_PREC_DF64))
    fail(FLZ_ERR_INVALID_ARG, "tensor-core reorthogonalization needs an FP64 basis (not the double-FP32 precision)");
  if (p.precision < FLZ_PREC_FP64 || p.precision > FLZ_PREC_FX64) fail(FLZ_ERR_INVALID_ARG, "bad precision");
  if (p.precision == FLZ_PREC_FX64 && p.recurrence != FLZ_REC_FORWARD)
    fail(FLZ_ERR_INVALID_ARG, "the fixed-point filter evaluates the forward recurrence only");
  flz_solver* s = new flz_solver();
  s->A = A;
  s->p = p;
  *out = s;
  FLZ_API_END
}

flz_status flz_solver_destroy(flz_solver* s) {
  FLZ_API_BEGIN
  delete s;
  FLZ_API_END
}

flz_status flz_solver_set_interval(flz_solver* s, double alpha, double beta) {
  FLZ_API_BEGIN
  if (!s || !(alpha < beta) || !std::isfinite(alpha) || !std::isfinite(beta)) fail(FLZ_ERR_INVALID_ARG, "need finite alpha < beta");
  s->alpha = alpha;
  s->beta = beta;
  s->has_interval = true;
  FLZ_API_END
}

flz_status flz_solver_set_start_vectors(flz_solver* s, const double* X, int64_t ld, int32_t cols,
                                        flz_memspace where) {
  FLZ_API_BEGIN
  if (!s || cols < 0 || (cols > 0 && !X)) fail(FLZ_ERR_INVALID_ARG, "bad arguments");
  if (where != FLZ_HOST && where != FLZ_DEVICE) fail(FLZ_ERR_INVALID_ARG, "bad memspace");
  const int64_t n = s->A->n;
  if (cols > 0 && ld < n) fail(FLZ_ERR_INVALID_ARG, "ld < n");
  if (s->p.precision == FLZ_PREC_DF64 && cols > 0)
    fail(FLZ_ERR_INVALID_ARG, "start vectors apply to solves with an FP64 basis (not the double-FP32 precision)");
  s->start_cols = 0;
  if (cols == 0) {
    s->start.release();
  } else {
    s->start.reserve((size_t)n * cols);
    FLZ_CUDA(cudaMemcpy2D(s->start.p, sizeof(double) * n, X, sizeof(double) * ld, sizeof(double) * n, (size_t)cols,
                          where == FLZ_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice));
    s->start_cols = cols;
  }
  FLZ_API_END
}

flz_status flz_solve(flz_solver* s, void* stream) {
  ::flz::clear_last_error();
  try {
    if (!s) fail(FLZ_ERR_INVALID_ARG, "solver is NULL");
    if (!s->has_interval) fail(FLZ_ERR_NO_INTERVAL, "set the interval first");
    const flz_status st = flz::solve(s, static_cast<cudaStream_t>(stream));
    if (st == FLZ_ERR_NOT_CONVERGED) flz::set_last_error("basis capacity reached before convergence; partial results");
    return st;
  } catch (const ::flz::Failure& f) {
    return f.status;
  } catch (const std::bad_alloc&) {
    ::flz::set_last_error("host allocation failed");
    return FLZ_ERR_OUT_OF_MEMORY;
  } catch (...) {
    ::flz::set_last_error("unexpected internal error");
    return FLZ_ERR_CUDA;
  }
}

flz_status flz_solve_sliced(flz_solver* s, int32_t nslices, void* stream) {
  ::flz::clear_last_error();
  try {
    if (!s) fail(FLZ_ERR_INVALID_ARG, "solver is NULL");
    if (!s->has_interval) fail(FLZ_ERR_NO_INTERVAL, "set the interval first");
    const flz_status st = flz::solve_sliced(s, nslices, static_cast<cudaStream_t>(stream));
    if (st == FLZ_ERR_NOT_CONVERGED) flz::set_last_error("a slice reached its basis capacity; partial results");
    return st;
  } catch (const ::flz::Failure& f) {
    return f.status;
  } catch (const std::bad_alloc&) {
    ::flz::set_last_error("host allocation failed");
    return FLZ_ERR_OUT_OF_MEMORY;
  } catch (...) {
    ::flz::set_last_error("unexpected internal error");
    return FLZ_ERR_CUDA;
  }
}

flz_status flz_get_count(const flz_solver* s, int64_t* count) {
  FLZ_API_BEGIN
  if (!s || !count) fail(FLZ_ERR_INVALID_ARG, "null argument");
  if (!s->solved) fail(FLZ_ERR_NOT_SOLVED, "no solve yet");
  *count = s->count;
  FLZ_API_END
}

flz_status flz_get_eigenvalues(const flz_solver* s, double* out, int64_t cap) {
  FLZ_API_BEGIN
  if (!s || (!out && s->count > 0)) fail(FLZ_ERR_INVALID_ARG, "null argument");
  if (!s->solved) fail(FLZ_ERR_NOT_SOLVED, "no solve yet");
  if (cap < s->count) fail(FLZ_ERR_CAPACITY, "need %lld slots", (long long)s->count);
  for (int64_t i = 0; i < s->count; ++i) out[i] = s->evals[i];
  FLZ_API_END
}

flz_status flz_get_residuals(const flz_solver* s, double* out, int64_t cap) {
  FLZ_API_BEGIN
  if (!s || (!out && s->count > 0)) fail(FLZ_ERR_INVALID_ARG, "null argument");
  if (!s->solved) fail(FLZ_ERR_NOT_SOLVED, "no solve yet");
  if (cap < s->count) fail(FLZ_ERR_CAPACITY, "need %lld slots", (long long)s->count);
  for (int64_t i = 0; i < s->count; ++i) out[i] = s->resid[i];
  FLZ_API_END
}

flz_status flz_get_eigenvectors(const flz_solver* s, double* out, int64_t ld, int64_t cap_cols, flz_memspace where) {
  FLZ_API_BEGIN
  if (!s || (!out && s->count > 0)) fail(FLZ_ERR_INVALID_ARG, "null argument");
  if (!s->solved) fail(FLZ_ERR_NOT_SOLVED, "no solve yet");
  const int64_t n = s->A->n;
  if (ld < n) fail(FLZ_ERR_INVALID_ARG, "ld < n");
  if (cap_cols < s->count) fail(FLZ_ERR_CAPACITY, "need %lld columns", (long long)s->count);
  if (where != FLZ_HOST && where != FLZ_DEVICE) fail(FLZ_ERR_INVALID_ARG, "bad memspace");
  if (s->count == 0) return FLZ_OK;
  const cudaMemcpyKind kind = where == FLZ_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  FLZ_CUDA(cudaMemcpy2D(out, sizeof(double) * ld, s->evecs.p, sizeof(double) * n, sizeof(double) * n,
                        (size_t)s->count, kind));
  FLZ_API_END
}

flz_status flz_get_checks(const flz_solver* s, flz_check* out, int64_t cap, int64_t* count) {
  FLZ_API_BEGIN
  if (!s || cap < 0 || (cap > 0 && !out)) fail(FLZ_ERR_INVALID_ARG, "bad arguments");
  const int64_t nc = (int64_t)s->checks.size();
  if (count) *count = nc;
  for (int64_t i = 0; i < std::min(cap, nc); ++i) out[i] = s->checks[i];
  FLZ_API_END
}

flz_status flz_get_stats(const flz_solver* s, flz_stats* out) {
  FLZ_API_BEGIN
  if (!s || !out) fail(FLZ_ERR_INVALID_ARG, "null argument");
  *out = s->stats;
  FLZ_API_END
}

}  // extern "C"
