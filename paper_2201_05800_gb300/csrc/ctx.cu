// C-ABI of libstdg: context, residual / Jv entry points and the Newton-Krylov
// slab solver (see include/stdg.h for the contract).
//
// Slab solve (Sec. 6.3, Newton-type nonlinear solver with a Krylov linear
// solver, as in the paper's 3D runs): U0 = 1 (x) u^n; while ||R(U)|| is above
// max(rtol ||R(U0)||, atol): solve J(U) dU = -R(U) by restarted GMRES(m) with
// classical Gram-Schmidt and selective re-orthogonalisation, Givens rotations
// on the host, matrix-free J v by the space-time operator kernel, right
// preconditioning by the point-block inverse P^-1 (precond.cuh) or left scaling
// by M_tau^-1; U += dU.  Then u^{n+1} = U^s (Eq. un).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "args_host.cuh"
#include "blas.cuh"
#include "common.cuh"
#include "lgl_host.h"
#include "ops.h"
#include "precond.cuh"
#include "stdg.h"

using namespace stdg;

namespace {

constexpr int kMaxGmresM = kMaxDots - 1;  // basis of m+1 vectors must fit one dot pass
constexpr size_t kSmemLimit = 227 * 1024;
constexpr int kSmall = 256;               // doubles of device / pinned scratch
constexpr int kProfClasses = 5;           // residual, Jv, Gram-Schmidt/vector, other, preconditioner

}  // namespace

struct stdg_ctx {
  stdg_config_desc d;
  cudaStream_t st = nullptr;
  int device = 0, sms = 0;
  int dim = 1, n = 2, s = 2, r = 1, nd = 1;
  long long nelem = 0;
  size_t state_len = 0, slab_len = 0;
  double h[3] = {1, 1, 1};
  OpArgs<double> a64;
  OpArgs<float> a32;
  int epb64[3] = {1, 1, 1};
  int epb32[3] = {1, 1, 1};
  int msp64[3] = {1, 1, 1};  // temporal split of the operator launches (OpArgs::msplit)
  int msp32[3] = {1, 1, 1};
  int nblk = 1;
  // FP32 buffers of the mixed-precision Krylov solve (STDG_MIXED_FP32 only)
  float *U32 = nullptr, *F032 = nullptr, *R32 = nullptr, *X32 = nullptr, *V32 = nullptr;
  // point-block preconditioner (STDG_PRECOND_POINT_BLOCK): P_I^-1 per spatial node, in the
  // working precision of the Krylov solve, and the preconditioned direction z = P^-1 v
  double* Pinv64 = nullptr;
  float *Pinv32 = nullptr, *Z32 = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  double *U = nullptr, *R = nullptr, *F0 = nullptr, *delta = nullptr, *uprev = nullptr;
  double *X1 = nullptr, *X2 = nullptr, *Xs = nullptr, *V = nullptr, *partials = nullptr, *small = nullptr;
  double* hpin = nullptr;
  double* rpart = nullptr;   // per-block norm sums of the residual kernel
  unsigned* errw = nullptr;  // error word of the kernels with bounded waits (0: none gave up)
  int nres_blocks = 1;
  double t = 0.0;
  bool have_slab = false;
  StageMatrix ext{};  // U0_m = sum_j ext[m][j] U_j of the previous slab (l_j(tau_m + 2))
  std::string err;
  // kernel timing (stdg_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_live;
  int prof_launches[kProfClasses] = {};
  double prof_ms[kProfClasses] = {};
};

namespace {

struct DevGuard {
  int prev = -1, dev;
  explicit DevGuard(int d) : dev(d) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
};

cudaEvent_t take_event(stdg_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Brackets one kernel launch with CUDA events when profiling is on.
struct Prof {
  stdg_ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  Prof(stdg_ctx* ctx, int k) : c(ctx), cls(k) {
    ++c->prof_launches[cls];  // counted whether or not timing is on
    if (c->prof && (a = take_event(c))) cudaEventRecord(a, c->st);
  }
  ~Prof() {
    if (!a) return;
    cudaEvent_t b = take_event(c);
    if (!b) {
      c->ev_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, c->st);
    c->ev_live.push_back({cls, {a, b}});
  }
};

// Sum the recorded launches (the stream must be synchronised) and recycle the events.
void prof_collect(stdg_ctx* c) {
  for (auto& x : c->ev_live) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, x.second.first, x.second.second) == cudaSuccess) {
      c->prof_ms[x.first] += ms;
    } else {
      cudaGetLastError();
    }
    c->ev_pool.push_back(x.second.first);
    c->ev_pool.push_back(x.second.second);
  }
  c->ev_live.clear();
}

stdg_status fail(stdg_ctx* c, stdg_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

#define CK(c, expr)                                                                                   \
  do {                                                                                                \
    cudaError_t _e = (expr);                                                                          \
    if (_e != cudaSuccess)                                                                            \
      return fail((c), STDG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));            \
  } while (0)

// CK inside a profiled bracket of class `cls`
#define PK(c, cls, expr)   \
  do {                     \
    Prof _p((c), (cls));   \
    CK((c), expr);         \
  } while (0)

#define CKS(expr)                        \
  do {                                   \
    stdg_status _s = (expr);             \
    if (_s != STDG_OK) return _s;        \
  } while (0)

int num_components(int eq, int dim) { return eq == STDG_EULER ? dim + 2 : 1; }

template <class T>
void fill_args(const stdg_ctx* c, OpArgs<T>& k) {
  fill_op_args<T>(k, c->dim, c->n, c->s, c->d.cells, c->h, c->d.dt, c->d.gamma, c->d.adv_vel, c->d.viscosity,
                  c->d.penalty);
}

stdg_status validate(const stdg_config_desc* d, std::string* why) {
  auto bad = [&](const char* m) { *why = m; return STDG_ERR_INVALID_ARG; };
  if (d->dim < 1 || d->dim > 3) return bad("dim must be 1..3");
  for (int a = 0; a < d->dim; ++a) {
    if (d->cells[a] < 1) return bad("cells must be >= 1");
    if (!(d->hi[a] > d->lo[a])) return bad("hi must exceed lo");
  }
  if (d->N < 1 || d->N > 7) return bad("N must be 1..7");
  if (d->s < 2 || d->s > 5) return bad("s must be 2..5");
  if (d->equation != STDG_ADVECTION && d->equation != STDG_EULER && d->equation != STDG_BURGERS)
    return bad("unknown equation");
  if (d->equation == STDG_BURGERS && d->dim > 2) return bad("Burgers is compiled for dim 1..2");
  if (d->flux != STDG_FLUX_RUSANOV) return bad("unknown flux");
  if (!(d->dt > 0) || !std::isfinite(d->dt)) return bad("dt must be positive");
  if (d->equation == STDG_EULER && !(d->gamma > 1.0)) return bad("gamma must exceed 1");
  if (d->precision != STDG_FP64 && d->precision != STDG_MIXED_FP32 && d->precision != STDG_MIXED_BF16)
    return bad("unknown precision");
  if (d->precision == STDG_MIXED_BF16 &&
      !(d->dim == 3 && d->equation == STDG_EULER && d->N == 3 && d->s == 3 && d->jv_mode == STDG_JV_EXACT))
    return bad("STDG_MIXED_BF16 is built for the 3D Euler N = 3, s = 3 shape with STDG_JV_EXACT");
  if (d->jv_mode != STDG_JV_FD && d->jv_mode != STDG_JV_EXACT) return bad("unknown jv_mode");
  if (d->newton_maxit < 1 || d->gmres_maxit < 1) return bad("maxit must be >= 1");
  if (d->gmres_m < 1 || d->gmres_m > kMaxGmresM) return bad("gmres_m must be 1..31");
  if (!(d->newton_rtol >= 0) || !(d->newton_atol >= 0) || !(d->gmres_rtol > 0)) return bad("bad tolerance");
  if (!(d->viscosity >= 0.0) || !std::isfinite(d->viscosity) || !std::isfinite(d->penalty))
    return bad("viscosity must be finite and >= 0");
  if (d->viscosity > 0.0 && d->equation == STDG_EULER) return bad("viscosity is supported for scalar equations");
  if (d->precond != STDG_PRECOND_NONE && d->precond != STDG_PRECOND_TEMPORAL_MASS &&
      d->precond != STDG_PRECOND_POINT_BLOCK)
    return bad("unknown precond");
  if (d->predictor != STDG_PREDICTOR_CONSTANT && d->predictor != STDG_PREDICTOR_EXTRAPOLATE)
    return bad("unknown predictor");
  return STDG_OK;
}

template <class T>
stdg_status alloc(stdg_ctx* c, T** p, size_t count) {
  size_t b = count * sizeof(T);
  if (c->d.hbm_budget_bytes && c->bytes + b > c->d.hbm_budget_bytes)
    return fail(c, STDG_ERR_OOM, "allocation exceeds hbm_budget_bytes");
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, STDG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  c->bytes += b;
  *p = static_cast<T*>(q);
  return STDG_OK;
}

// Elements per CTA (epb) and temporal split (msplit) of the operator kernel.  The
// kernel is throughput bound per SM, so its time follows the most loaded SM: the work
// units are (element, temporal node) pairs and a CTA holds epb * s / msplit of them.
// For the FP64 FD Jacobian-vector product (FP64-pipe bound), when the element tiles give
// fewer than 32 warps per SM (the residency of these 64-register kernels), each CTA takes
// one temporal node of its tile (msplit = s): s times as many CTAs, each with 1/s of the
// work, so that the resident warps keep the FP64 pipe busy through the barriers (measured
// on the 64^2 vortex: 0.137 -> 0.133 ms per launch).  The FP32 exact product (latency
// bound) and the residual with its norms were slower split (27.1 -> 27.9 us, +5%).
// Score = load balance x active lanes x a small bonus for faces shared inside a CTA;
// CTAs are limited by shared memory (228 KB per SM, 1 KB reserved per CTA), threads
// (2048 per SM) and 32 CTAs per SM.
int choose_epb(const stdg_ctx* c, int mode, size_t tsize, int* msplit) {
  int best = 1, best_ms = 1;
  double best_score = -1.0;
  const int max_epb = std::max(1, 256 / c->nd);
  for (int epb = 1; epb <= max_epb && epb <= c->nelem; ++epb) {
    const size_t smem = operator_smem_bytes(c->dim, c->r, tsize, mode, c->n, c->s, epb);
    if (smem > kSmemLimit) break;
    int threads = std::min(256, epb * c->nd);
    threads = (threads + 31) / 32 * 32;
    const int bps = std::min({(int)(233472 / (smem + 1024)), 2048 / threads, 32});
    if (bps < 1) break;
    const long long tiles = (c->nelem + epb - 1) / epb;
    const bool may_split = mode == kModeJvFD && tsize == sizeof(double);
    const int ms = may_split && tiles * (threads / 32) < 32LL * c->sms ? c->s : 1;
    const long long nblocks = tiles * ms;
    const long long per_sm = (nblocks + c->sms - 1) / c->sms;
    const double balance =
        ((double)c->nelem * c->s / c->sms) / ((double)per_sm * epb * ((double)c->s / ms));
    // idle lanes cost little in a kernel bound by the per-SM FP64 pipe: weigh them half
    const double lanes = (double)std::min(epb * c->nd, 256) / threads;
    const double score = balance * (0.5 + 0.5 * lanes) * (1.0 + 0.1 * (epb - 1) / epb);
    if (score > best_score + 1e-9) {
      best_score = score;
      best = epb;
      best_ms = ms;
    }
  }
  *msplit = best_ms;
  return best;
}

// ---- operator launches
stdg_status op_residual(stdg_ctx* c, const double* U, const double* uprev, double* out, double* fout) {
  OpArgs<double> k = c->a64;
  k.epb = c->epb64[kModeResidual];
  k.msplit = c->msp64[kModeResidual];
  k.U = U;
  k.uprev = uprev;
  k.out = out;
  k.fout = fout;
  Prof p(c, 0);
  CK(c, launch_operator<double>(c->dim, c->d.equation, kModeResidual, k, c->st));
  return STDG_OK;
}

// Buffers and constants of one working precision of the Krylov solve: FP64
// (plain path) or FP32 (STDG_MIXED_FP32, Newton stays FP64).
template <class T>
struct KView {
  const OpArgs<T>* args;
  const int* epb;
  const int* msp;
  T* U;   // Newton iterate in T
  T* F0;  // F(U) in T (FD Jv)
  T* R;   // Newton residual in T
  T* X;   // slab scratch in T
  T* V;   // Krylov basis, gmres_m + 1 rows
  T* Z;   // preconditioned direction P^-1 v (point-block preconditioner)
  T* Pinv;  // P_I^-1 per spatial node (point-block preconditioner)
};

KView<double> view(stdg_ctx* c, double*) {
  return {&c->a64, c->epb64, c->msp64, c->U, c->F0, c->R, c->X1, c->V, c->X2, c->Pinv64};
}
KView<float> view(stdg_ctx* c, float*) {
  return {&c->a32, c->epb32, c->msp32, c->U32, c->F032, c->R32, c->X32, c->V32, c->Z32, c->Pinv32};
}

// F(U) only, in precision T (FD Jv base point of the mixed path)
template <class T>
stdg_status op_spatial(stdg_ctx* c, const KView<T>& kv, const T* U, T* fout) {
  OpArgs<T> k = *kv.args;
  k.epb = kv.epb[kModeResidual];
  k.msplit = kv.msp[kModeResidual];
  k.U = U;
  k.uprev = nullptr;
  k.out = nullptr;
  k.fout = fout;
  Prof p(c, 0);
  CK(c, launch_operator<T>(c->dim, c->d.equation, kModeResidual, k, c->st));
  return STDG_OK;
}

// lscale: rows of temporal node m divided by omega_m (the GMRES left scaling of
// STDG_PRECOND_TEMPORAL_MASS); the public stdg_jv always returns J v unscaled.
template <class T>
stdg_status op_jv_t(stdg_ctx* c, const KView<T>& kv, const T* U, const T* F0, const T* v, double vscale,
                    double eps, T* out, bool lscale) {
  const int mode = c->d.jv_mode == STDG_JV_EXACT ? kModeJvExact : kModeJvFD;
  OpArgs<T> k = *kv.args;
  k.epb = kv.epb[mode];
  k.msplit = kv.msp[mode];
  k.U = U;
  k.v = v;
  k.F0 = F0;
  k.vscale = (T)vscale;
  k.eps = (T)eps;
  k.inv_eps = eps > 0.0 ? (T)(1.0 / eps) : (T)0;
  k.lscale = lscale ? 1 : 0;
  k.out = out;
  k.err = c->errw;
  Prof p(c, 1);
  if constexpr (std::is_same<T, float>::value) {
    if (mode == kModeJvExact) {
      bool handled = false;
      CK(c, launch_jv_tangent(c->dim, c->d.equation, k, c->st, &handled, c->d.precision == STDG_MIXED_BF16));
      if (handled) return STDG_OK;
    }
  }
  CK(c, launch_operator<T>(c->dim, c->d.equation, mode, k, c->st));
  return STDG_OK;
}

// The error word of the bounded waits: STDG_ERR_TIMEOUT if a kernel gave up waiting for its
// staged data (its outputs are then incomplete).  Synchronises the stream.
stdg_status check_errw(stdg_ctx* c) {
  unsigned h = 0;
  CK(c, cudaMemcpyAsync(&h, c->errw, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (h) {
    cudaMemsetAsync(c->errw, 0, sizeof(unsigned), c->st);
    return fail(c, STDG_ERR_TIMEOUT, "a kernel's bounded wait for its staged tile ran out");
  }
  return STDG_OK;
}

stdg_status op_jv(stdg_ctx* c, const double* U, const double* F0, const double* v, double vscale, double eps,
                  double* out, bool lscale = false) {
  return op_jv_t<double>(c, view(c, (double*)nullptr), U, F0, v, vscale, eps, out, lscale);
}

// ---- reductions
template <class T>
stdg_status dots_to_small(stdg_ctx* c, const T* V, int k, const T* w, int small_off) {
  int used = c->nblk;
  PK(c, 2, (multidot<T, T>(V, c->slab_len, k, w, c->slab_len, c->partials, c->nblk, c->st, &used)));
  PK(c, 2, reduce_partials(c->partials, used, k, c->small + small_off, c->st));
  return STDG_OK;
}

stdg_status fetch_small(stdg_ctx* c, int off, int count) {
  CK(c, cudaMemcpyAsync(c->hpin + off, c->small + off, count * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  return STDG_OK;
}

template <class T>
stdg_status norm2(stdg_ctx* c, const T* x, size_t L, double* out) {
  int used = c->nblk;
  PK(c, 2, (multidot<T, T>(x, L, 1, x, L, c->partials, c->nblk, c->st, &used)));
  PK(c, 2, reduce_partials(c->partials, used, 1, c->small + 200, c->st));
  CKS(fetch_small(c, 200, 1));
  *out = std::sqrt(c->hpin[200]);
  return STDG_OK;
}

// Residual of the Newton iterate with its norms from the same pass: returns |R|_2, |U|_2 and
// |W^-1 R|_2 (W = M_tau with the left temporal-mass scaling, else I) and writes W^-1 R as the
// first Krylov vector (v0d in FP64 or v0f in FP32, either may be null).
stdg_status op_residual_norms(stdg_ctx* c, double* v0d, float* v0f, double* res, double* unorm, double* b0) {
  OpArgs<double> k = c->a64;
  k.epb = c->epb64[kModeResidual];
  k.msplit = c->msp64[kModeResidual];
  k.U = c->U;
  k.uprev = c->uprev;
  k.out = c->R;
  k.fout = c->F0;
  k.nrm = c->rpart;
  k.nrm_stride = kPartialStride;
  k.v0w = c->d.precond == STDG_PRECOND_TEMPORAL_MASS ? 1 : 0;
  k.v0d = v0d;
  k.v0f = v0f;
  {
    Prof p(c, 0);
    CK(c, launch_operator<double>(c->dim, c->d.equation, kModeResidual, k, c->st));
  }
  PK(c, 2, reduce_partials(c->rpart, c->nres_blocks, 3, c->small + 210, c->st));
  CKS(fetch_small(c, 210, 3));
  *res = std::sqrt(c->hpin[210]);
  *unorm = std::sqrt(c->hpin[211]);
  *b0 = std::sqrt(c->hpin[212]);
  return STDG_OK;
}

// delta as the T-typed input of a Jacobian-vector product (the FP32 copy lives in X)
template <class T> const T* delta_in(stdg_ctx* c, T* X);
template <> const double* delta_in<double>(stdg_ctx* c, double*) { return c->delta; }
template <> const float* delta_in<float>(stdg_ctx*, float* X) { return X; }

template <class T> double fd_base_eps();
template <> double fd_base_eps<double>() { return std::sqrt(2.220446049250313e-16); }
template <> double fd_base_eps<float>() { return std::sqrt(1.1920928955078125e-07); }

// ---- GMRES(m) for J(U) delta = -R, delta (FP64) accumulated in c->delta.
//
// Arnoldi with classical Gram-Schmidt and a selective re-orthogonalisation
// test: one fused pass gives p_i = V_i . w (i <= j) and |w|^2 (w is the row
// after the basis); |w - V h|^2 = |w|^2 - |h|^2 (Pythagoras); a second
// projection is made only when that norm fell below |w|/10 (strong
// cancellation; the classical DGKS bound 1/sqrt(2) fired in most steps of the
// left-scaled system without changing iteration counts or the true residual).
// Basis rows are stored unnormalised with scale factors sig_i
// (v_i = sig_i V_i), so no scaling pass is needed; coefficients reach the
// update kernel by value.  Hessenberg, Givens rotations and the triangular
// solve are FP64 on the host in both precisions; the basis, the Jacobian-
// vector products and the per-thread sums of the dot passes are in T.
template <class T>
stdg_status gmres(stdg_ctx* c, double eps_u, double beta_pre, int* its_out, int* jv_out) {
  const KView<T> kv = view(c, (T*)nullptr);
  const int m = c->d.gmres_m;
  const size_t L = c->slab_len;
  const bool ls = c->d.precond == STDG_PRECOND_TEMPORAL_MASS;
  const bool pb = c->d.precond == STDG_PRECOND_POINT_BLOCK;
  const int blk = c->nd * c->r;
  TimeWeights winv;  // left scaling of the rows of temporal node m (1 without preconditioning)
  for (int q = 0; q < 8; ++q) winv.w[q] = (ls && q < c->s) ? 1.0 / (double)c->a64.omega[q] : 1.0;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m), sig(m + 1);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  auto Vrow = [&](int i) { return kv.V + (size_t)i * L; };
  CK(c, cudaMemsetAsync(c->delta, 0, L * sizeof(double), c->st));
  // the Newton residual in T (a cast for the mixed path), then b = -(M^-1 (x) I) R (or -R)
  if (!std::is_same<T, double>::value)
    PK(c, 2, (scale_add<double, T>(kv.R, c->R, 1.0, nullptr, 0.0, L, c->st)));
  // V_0 = (M^-1 (x) I) R (or R): written with its norm by the residual kernel when beta_pre >= 0
  double beta0 = beta_pre;
  if (beta_pre < 0.0) {
    PK(c, 2, (tnode_scale_add<T>(Vrow(0), kv.R, 1.0, winv, nullptr, 0.0, c->nelem, c->s, blk, c->st)));
    CKS(norm2<T>(c, Vrow(0), L, &beta0));
  }
  const double tol = c->d.gmres_rtol * beta0;
  int its = 0, jvs = 0;
  bool first = true;
  while (its < c->d.gmres_maxit && beta0 > 0.0) {
    double beta;
    if (first) {
      beta = beta0;
      sig[0] = -1.0 / beta0;  // v_0 = b / |b|, V_0 holds -b
    } else {
      // restart: V_0 = -(b - J delta) with delta cast to T
      double nd;
      CKS(norm2<double>(c, c->delta, L, &nd));
      if (!std::is_same<T, double>::value)
        PK(c, 2, (scale_add<double, T>(kv.X, c->delta, 1.0, nullptr, 0.0, L, c->st)));
      const T* dT = delta_in<T>(c, kv.X);
      CKS(op_jv_t<T>(c, kv, kv.U, kv.F0, dT, 1.0, eps_u / (nd > 0 ? nd : 1.0), Vrow(0), ls));
      ++jvs;
      PK(c, 2, (tnode_scale_add<T>(Vrow(0), kv.R, -1.0, winv, Vrow(0), -1.0, c->nelem, c->s, blk, c->st)));
      CKS(norm2<T>(c, Vrow(0), L, &beta));
      if (!(beta > tol)) break;
      sig[0] = 1.0 / beta;
    }
    first = false;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int kdim = 0;
    bool done = false;
    for (int j = 0; j < m && its < c->d.gmres_maxit; ++j) {
      T* w = Vrow(j + 1);
      if (pb) {
        // right preconditioning: w = J z with z = P^-1 v_j (|v_j| = 1, so the FD step
        // eps_u / |v_j| is kept; |z| is within the norm bounds of P^-1)
        PK(c, 4, (pb_apply<T, T, T>(kv.Z, Vrow(j), sig[j], kv.Pinv, 0, c->nelem, c->s, c->nd, c->r, c->st)));
        CKS(op_jv_t<T>(c, kv, kv.U, kv.F0, kv.Z, 1.0, eps_u, w, false));
      } else {
        CKS(op_jv_t<T>(c, kv, kv.U, kv.F0, Vrow(j), sig[j], eps_u, w, ls));
      }
      ++jvs;
      // p_i = V_i . w (i <= j) and |w|^2 in one pass over rows 0..j+1
      CKS(dots_to_small<T>(c, kv.V, j + 2, w, 0));
      CKS(fetch_small(c, 0, j + 2));
      double w2 = c->hpin[j + 1], h2 = 0.0;
      Coefs cf;
      for (int i = 0; i <= j; ++i) {
        Hij(i, j) = sig[i] * c->hpin[i];
        h2 += Hij(i, j) * Hij(i, j);
        cf.c[i] = sig[i] * Hij(i, j);
      }
      PK(c, 2, (update<T, T>(w, kv.V, L, j + 1, cf, L, c->st)));
      double r2 = w2 - h2;
      if (!(r2 > 0.01 * w2)) {
        // strong cancellation: project once more and take the norm directly
        CKS(dots_to_small<T>(c, kv.V, j + 2, w, 0));
        CKS(fetch_small(c, 0, j + 2));
        double e2 = 0.0;
        for (int i = 0; i <= j; ++i) {
          double hi = sig[i] * c->hpin[i];
          Hij(i, j) += hi;
          e2 += hi * hi;
          cf.c[i] = sig[i] * hi;
        }
        PK(c, 2, (update<T, T>(w, kv.V, L, j + 1, cf, L, c->st)));
        r2 = c->hpin[j + 1] - e2;
      }
      if (!std::isfinite(r2) || !std::isfinite(w2)) return fail(c, STDG_ERR_NAN, "GMRES: non-finite Krylov vector");
      const double hn = std::sqrt(r2 > 0.0 ? r2 : 0.0);
      // apply the previous rotations to the new column, then a new one
      for (int i = 0; i < j; ++i) {
        double t0 = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t0;
      }
      double den = std::hypot(Hij(j, j), hn);
      if (den == 0.0) den = 1e-300;
      cs[j] = Hij(j, j) / den;
      sn[j] = hn / den;
      Hij(j, j) = den;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      kdim = j + 1;
      sig[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
      if (std::fabs(g[j + 1]) <= tol || hn <= 1e-300 * beta0) {
        done = true;
        break;
      }
    }
    // y = H^-1 g (upper triangular), delta += sum_i y_i sig_i V_i
    for (int i = kdim - 1; i >= 0; --i) {
      double acc = g[i];
      for (int q = i + 1; q < kdim; ++q) acc -= Hij(i, q) * y[q];
      y[i] = acc / Hij(i, i);
    }
    if (kdim > 0) {
      Coefs cf;
      for (int i = 0; i < kdim; ++i) cf.c[i] = -y[i] * sig[i];
      if (pb) {
        // delta += P^-1 (sum_i y_i v_i), the sum formed in the scratch row X
        CK(c, cudaMemsetAsync(kv.X, 0, L * sizeof(T), c->st));
        PK(c, 2, (update<T, T>(kv.X, kv.V, L, kdim, cf, L, c->st)));
        PK(c, 4, (pb_apply<T, T, double>(c->delta, kv.X, 1.0, kv.Pinv, 1, c->nelem, c->s, c->nd, c->r, c->st)));
      } else {
        PK(c, 2, (update<T, double>(c->delta, kv.V, L, kdim, cf, L, c->st)));
      }
    }
    if (done) break;
  }
  *its_out = its;
  *jv_out = jvs;
  return STDG_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void stdg_config_default(stdg_config_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->dim = 1;
  d->cells[0] = d->cells[1] = d->cells[2] = 16;
  for (int a = 0; a < 3; ++a) {
    d->lo[a] = 0.0;
    d->hi[a] = 1.0;
  }
  d->N = 3;
  d->s = 3;
  d->equation = STDG_ADVECTION;
  d->adv_vel[0] = 1.0;
  d->gamma = 1.4;
  d->flux = STDG_FLUX_RUSANOV;
  d->dt = 0.01;
  d->precision = STDG_FP64;
  d->jv_mode = STDG_JV_FD;
  d->newton_rtol = 1e-10;
  d->newton_atol = 0.0;
  d->newton_maxit = 20;
  d->gmres_m = 30;
  d->gmres_rtol = 1e-3;
  d->gmres_maxit = 300;
  d->hbm_budget_bytes = 0;
  d->precond = STDG_PRECOND_TEMPORAL_MASS;
  d->predictor = STDG_PREDICTOR_CONSTANT;
}

stdg_status stdg_create(const stdg_config_desc* desc, void* cuda_stream, stdg_ctx** out) {
  if (!out) return STDG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return STDG_ERR_INVALID_ARG;
  std::string why;
  if (validate(desc, &why) != STDG_OK) return STDG_ERR_INVALID_ARG;
  const bool mixed = desc->precision != STDG_FP64;
  stdg_ctx* c = new stdg_ctx();
  c->d = *desc;
  c->st = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return STDG_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (c->sms <= 0) c->sms = 1;
  c->dim = desc->dim;
  c->n = desc->N + 1;
  c->s = desc->s;
  c->r = num_components(desc->equation, desc->dim);
  c->nd = 1;
  c->nelem = 1;
  for (int a = 0; a < c->dim; ++a) {
    c->nd *= c->n;
    c->nelem *= desc->cells[a];
    c->h[a] = (desc->hi[a] - desc->lo[a]) / desc->cells[a];
  }
  c->state_len = (size_t)c->nelem * c->nd * c->r;
  c->slab_len = c->state_len * c->s;
  fill_args(c, c->a64);
  fill_args(c, c->a32);
  {
    // Lagrange basis of the temporal LGL nodes evaluated one slab later: l_j(tau_m + 2)
    double E[64];
    lagrange_shift_matrix(c->s, 2.0, E);
    for (int m = 0; m < c->s; ++m)
      for (int j = 0; j < c->s; ++j) c->ext.a[m][j] = E[m * c->s + j];
  }
  for (int mode = 0; mode < 3; ++mode) {
    c->epb64[mode] = choose_epb(c, mode, sizeof(double), &c->msp64[mode]);
    c->epb32[mode] = choose_epb(c, mode, sizeof(float), &c->msp32[mode]);
    if (operator_smem_bytes(c->dim, c->r, sizeof(double), mode, c->n, c->s, c->epb64[mode]) > kSmemLimit) {
      delete c;
      return STDG_ERR_UNSUPPORTED;
    }
  }
  c->nblk = 4 * c->sms;
  c->nres_blocks = (int)((c->nelem + c->epb64[kModeResidual] - 1) / c->epb64[kModeResidual]) *
                   c->msp64[kModeResidual];
  const size_t L = c->slab_len, S = c->state_len;
  const size_t nbasis = L * (size_t)(desc->gmres_m + 1);
  const bool pbp = desc->precond == STDG_PRECOND_POINT_BLOCK;
  const size_t npinv = (size_t)c->nelem * c->nd * c->s * c->s;
  stdg_status st = STDG_OK;
  if ((st = alloc(c, &c->U, L)) || (st = alloc(c, &c->R, L)) || (st = alloc(c, &c->F0, L)) ||
      (st = alloc(c, &c->delta, L)) || (st = alloc(c, &c->X1, L)) || (st = alloc(c, &c->X2, L)) ||
      (st = alloc(c, &c->uprev, S)) || (st = alloc(c, &c->Xs, S)) ||
      (!mixed && (st = alloc(c, &c->V, nbasis))) ||
      (mixed && ((st = alloc(c, &c->U32, L)) || (st = alloc(c, &c->F032, L)) || (st = alloc(c, &c->R32, L)) ||
                 (st = alloc(c, &c->X32, L)) || (st = alloc(c, &c->V32, nbasis)))) ||
      (pbp && !mixed && (st = alloc(c, &c->Pinv64, npinv))) ||
      (pbp && mixed && ((st = alloc(c, &c->Pinv32, npinv)) || (st = alloc(c, &c->Z32, L)))) ||
      (st = alloc(c, &c->partials, (size_t)c->nblk * kPartialStride)) || (st = alloc(c, &c->small, kSmall)) ||
      (st = alloc(c, &c->rpart, (size_t)c->nres_blocks * kPartialStride)) || (st = alloc(c, &c->errw, 4))) {
    stdg_destroy(c);
    return st;
  }
  if (cudaMallocHost(&c->hpin, kSmall * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->hpin = nullptr;
    stdg_destroy(c);
    return STDG_ERR_OOM;
  }
  if (cudaMemsetAsync(c->errw, 0, 4 * sizeof(unsigned), c->st) != cudaSuccess ||
      cudaMemsetAsync(c->uprev, 0, S * sizeof(double), c->st) != cudaSuccess ||
      cudaMemsetAsync(c->U, 0, L * sizeof(double), c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess) {
    cudaGetLastError();
    stdg_destroy(c);
    return STDG_ERR_CUDA;
  }
  *out = c;
  return STDG_OK;
}

stdg_status stdg_destroy(stdg_ctx* c) {
  if (!c) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  cudaStreamSynchronize(c->st);
  prof_collect(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->hpin) cudaFreeHost(c->hpin);
  cudaGetLastError();
  delete c;
  return STDG_OK;
}

size_t stdg_state_len(const stdg_ctx* c) { return c ? c->state_len : 0; }
size_t stdg_slab_len(const stdg_ctx* c) { return c ? c->slab_len : 0; }
size_t stdg_coord_len(const stdg_ctx* c) { return c ? (size_t)c->nelem * c->nd * c->dim : 0; }
size_t stdg_device_bytes(const stdg_ctx* c) { return c ? c->bytes : 0; }

stdg_status stdg_node_coordinates(const stdg_ctx* cc, double* X, int kind) {
  stdg_ctx* c = const_cast<stdg_ctx*>(cc);
  if (!c || !X || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  double xi[16], w[16];
  lgl_rule(c->n, xi, w);
  std::vector<double> h((size_t)c->nelem * c->nd * c->dim);
  const int K0 = c->d.cells[0], K1 = c->dim > 1 ? c->d.cells[1] : 1;
  for (long long e = 0; e < c->nelem; ++e) {
    long long ec[3] = {e % K0, (e / K0) % K1, e / ((long long)K0 * K1)};
    for (int node = 0; node < c->nd; ++node) {
      int idx[3] = {node % c->n, (node / c->n) % c->n, node / (c->n * c->n)};
      for (int a = 0; a < c->dim; ++a)
        h[((size_t)e * c->nd + node) * c->dim + a] =
            c->d.lo[a] + c->h[a] * ((double)ec[a] + 0.5 * (1.0 + xi[idx[a]]));
    }
  }
  if (kind == STDG_HOST) {
    std::memcpy(X, h.data(), h.size() * sizeof(double));
  } else {
    CK(c, cudaMemcpyAsync(X, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return STDG_OK;
}

stdg_status stdg_set_state(stdg_ctx* c, const double* u, int kind) {
  if (!c || !u || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  CK(c, cudaMemcpyAsync(c->uprev, u, c->state_len * sizeof(double),
                        kind == STDG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->st));
  if (kind == STDG_HOST) CK(c, cudaStreamSynchronize(c->st));
  c->have_slab = false;
  return STDG_OK;
}

stdg_status stdg_get_state(const stdg_ctx* cc, double* u, int kind) {
  stdg_ctx* c = const_cast<stdg_ctx*>(cc);
  if (!c || !u || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  CK(c, cudaMemcpyAsync(u, c->uprev, c->state_len * sizeof(double),
                        kind == STDG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
  if (kind == STDG_HOST) CK(c, cudaStreamSynchronize(c->st));
  return STDG_OK;
}

stdg_status stdg_get_slab(const stdg_ctx* cc, double* U, int kind) {
  stdg_ctx* c = const_cast<stdg_ctx*>(cc);
  if (!c || !U || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  if (!c->have_slab) return fail(c, STDG_ERR_INVALID_ARG, "no slab has been solved since the last set_state");
  DevGuard g(c->device);
  CK(c, cudaMemcpyAsync(U, c->U, c->slab_len * sizeof(double),
                        kind == STDG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
  if (kind == STDG_HOST) CK(c, cudaStreamSynchronize(c->st));
  return STDG_OK;
}

stdg_status stdg_residual(stdg_ctx* c, const double* U, const double* uprev, double* R, int kind) {
  if (!c || !U || !uprev || !R || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  if (kind == STDG_DEVICE) return op_residual(c, U, uprev, R, nullptr);
  CK(c, cudaMemcpyAsync(c->X1, U, c->slab_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(c, cudaMemcpyAsync(c->Xs, uprev, c->state_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CKS(op_residual(c, c->X1, c->Xs, c->X2, nullptr));
  CK(c, cudaMemcpyAsync(R, c->X2, c->slab_len * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  return STDG_OK;
}

stdg_status stdg_jv(stdg_ctx* c, const double* U, const double* uprev, const double* v, double* Jv, int kind) {
  (void)uprev;
  if (!c || !U || !v || !Jv || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  const double* dU = U;
  const double* dv = v;
  double* dout = Jv;
  if (kind == STDG_HOST) {
    CK(c, cudaMemcpyAsync(c->X1, U, c->slab_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->X2, v, c->slab_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
    dU = c->X1;
    dv = c->X2;
    dout = c->R;
  }
  double eps = 0.0;
  if (c->d.jv_mode == STDG_JV_FD) {
    double nu, nv;
    CKS(norm2<double>(c, dU, c->slab_len, &nu));
    CKS(norm2<double>(c, dv, c->slab_len, &nv));
    eps = fd_base_eps<double>() * (1.0 + nu) / (nv > 0 ? nv : 1.0);
    CKS(op_residual(c, dU, c->uprev, nullptr, c->F0));
  }
  CKS(op_jv(c, dU, c->F0, dv, 1.0, eps, dout));
  if (kind == STDG_HOST) {
    CK(c, cudaMemcpyAsync(Jv, dout, c->slab_len * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return STDG_OK;
}

stdg_status stdg_slab_norm(stdg_ctx* c, const double* x, int kind, double* out) {
  if (!c || !x || !out || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  const double* dx = x;
  if (kind == STDG_HOST) {
    CK(c, cudaMemcpyAsync(c->X1, x, c->slab_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
    dx = c->X1;
  }
  return norm2<double>(c, dx, c->slab_len, out);
}

stdg_status stdg_advance_slab(stdg_ctx* c, stdg_slab_stats* stats) {
  if (!c) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  stdg_slab_stats S;
  std::memset(&S, 0, sizeof(S));
  const size_t L = c->slab_len;
  const int blk = c->nd * c->r;
  // extrapolated guess from the previous slab (kept in X1 until the constant guess is scored)
  const bool extrap = c->d.predictor == STDG_PREDICTOR_EXTRAPOLATE && c->have_slab;
  if (extrap) PK(c, 3, temporal_mix(c->X1, c->U, c->ext, c->nelem, c->s, blk, c->st));
  PK(c, 3, broadcast_slab<double>(c->U, c->uprev, c->nelem, c->s, blk, c->st));
  const bool mixed0 = c->d.precision != STDG_FP64;
  // the residual kernel also writes the first Krylov vector into the basis of the working
  // precision and returns |R|, |U| (FD step) and that vector's norm
  double* v0d = mixed0 ? nullptr : c->V;
  float* v0f = mixed0 ? c->V32 : nullptr;
  double res, unorm, b0;
  CKS(op_residual_norms(c, v0d, v0f, &res, &unorm, &b0));
  ++S.residual_evals;
  S.res0 = res;
  // the target is relative to the constant guess whichever iterate the solve starts from
  const double target = std::fmax(c->d.newton_rtol * res, c->d.newton_atol);
  if (extrap && res > target) {
    CK(c, cudaMemcpyAsync(c->U, c->X1, L * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    double res_e, unorm_e, b0_e;
    CKS(op_residual_norms(c, v0d, v0f, &res_e, &unorm_e, &b0_e));
    ++S.residual_evals;
    if (std::isfinite(res_e) && res_e < res) {
      res = res_e;
      unorm = unorm_e;
      b0 = b0_e;
    } else {
      // the extrapolation is worse: back to the constant guess
      PK(c, 3, broadcast_slab<double>(c->U, c->uprev, c->nelem, c->s, blk, c->st));
      CKS(op_residual_norms(c, v0d, v0f, &res, &unorm, &b0));
      ++S.residual_evals;
    }
  }
  const bool mixed = c->d.precision != STDG_FP64;
  stdg_status status = STDG_OK;
  while (true) {
    if (!std::isfinite(res)) {
      status = fail(c, STDG_ERR_NAN, "Newton: non-finite residual norm");
      break;
    }
    if (res <= target) break;
    if (S.newton_its >= c->d.newton_maxit) {
      status = fail(c, STDG_ERR_NOT_CONVERGED, "Newton: newton_maxit reached");
      break;
    }
    const double nu = unorm;
    int its = 0, jvs = 0;
    if (c->d.precond == STDG_PRECOND_POINT_BLOCK) {
      if (mixed) PK(c, 4, (pb_build<float>(c->dim, c->d.equation, c->a64, c->U, c->Pinv32, c->st)));
      else PK(c, 4, (pb_build<double>(c->dim, c->d.equation, c->a64, c->U, c->Pinv64, c->st)));
    }
    if (mixed) {
      // inner solve in FP32 around the FP32 copy of the Newton iterate; the
      // FP64 residual below refines (iterative refinement)
      PK(c, 2, (scale_add<double, float>(c->U32, c->U, 1.0, nullptr, 0.0, L, c->st)));
      if (c->d.jv_mode == STDG_JV_FD) CKS(op_spatial<float>(c, view(c, (float*)nullptr), c->U32, c->F032));
      CKS(gmres<float>(c, fd_base_eps<float>() * (1.0 + nu), b0, &its, &jvs));
    } else {
      CKS(gmres<double>(c, fd_base_eps<double>() * (1.0 + nu), b0, &its, &jvs));
    }
    S.gmres_its += its;
    S.jv_evals += jvs;
    PK(c, 2, (scale_add<double, double>(c->U, c->U, 1.0, c->delta, 1.0, L, c->st)));
    CKS(op_residual_norms(c, v0d, v0f, &res, &unorm, &b0));
    ++S.residual_evals;
    ++S.newton_its;
  }
  S.res_final = res;
  if (status == STDG_OK) {
    const stdg_status we = check_errw(c);
    if (we != STDG_OK) status = we;
  }
  if (status != STDG_ERR_NAN) {
    PK(c, 3, extract_last<double>(c->uprev, c->U, c->nelem, c->s, blk, c->st));
    c->t += c->d.dt;
    c->have_slab = true;
  }
  CK(c, cudaStreamSynchronize(c->st));
  prof_collect(c);
  if (stats) *stats = S;
  return status;
}

stdg_status stdg_spatial_operator(stdg_ctx* c, const double* U, double* F, int kind) {
  if (!c || !U || !F || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  if (kind == STDG_DEVICE) return op_residual(c, U, c->uprev, nullptr, F);
  CK(c, cudaMemcpyAsync(c->X1, U, c->slab_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CKS(op_residual(c, c->X1, c->uprev, nullptr, c->X2));
  CK(c, cudaMemcpyAsync(F, c->X2, c->slab_len * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  return STDG_OK;
}

stdg_status stdg_jv_fp32(stdg_ctx* c, const float* U, const float* v, float* Jv) {
  if (!c || !U || !v || !Jv) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  const int saved = c->d.jv_mode;
  c->d.jv_mode = STDG_JV_EXACT;
  const stdg_status st = op_jv_t<float>(c, view(c, (float*)nullptr), U, nullptr, v, 1.0, 0.0, Jv, false);
  c->d.jv_mode = saved;
  if (st != STDG_OK) return st;
  return check_errw(c);
}

stdg_status stdg_jv_fd_apply(stdg_ctx* c, const double* U, const double* F0, const double* v, double eps,
                             double* Jv) {
  if (!c || !U || !F0 || !v || !Jv || !(eps > 0.0)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  OpArgs<double> k = c->a64;
  k.epb = c->epb64[kModeJvFD];
  k.msplit = c->msp64[kModeJvFD];
  k.U = U;
  k.v = v;
  k.F0 = F0;
  k.vscale = 1.0;
  k.eps = eps;
  k.inv_eps = 1.0 / eps;
  k.out = Jv;
  Prof p(c, 1);
  CK(c, launch_operator<double>(c->dim, c->d.equation, kModeJvFD, k, c->st));
  return STDG_OK;
}

stdg_status stdg_lodg_residual(stdg_ctx* c, const double* U, const double* uprev, double* R, int form,
                               int kind) {
  if (!c || !U || !uprev || !R || (form != 0 && form != 1) || (kind != STDG_HOST && kind != STDG_DEVICE))
    return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  // Lobatto IIIC matrix from the temporal DG-SEM matrices (Eq. SBP_to_RK):
  // A = 1/2 Dtilde^-1, Dtilde = D_tau + M_tau^-1 e_1 e_1^T; the A^-1 form uses 2 Dtilde
  const int s = c->s;
  double tau[16], om[16], Dt[256];
  lgl_rule(s, tau, om);
  diff_matrix(s, tau, Dt);
  double W[kMaxS][2 * kMaxS];
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      W[i][j] = Dt[i * s + j] + (i == 0 && j == 0 ? 1.0 / om[0] : 0.0);
      W[i][s + j] = i == j ? 1.0 : 0.0;
    }
  StageMatrix A;
  std::memset(&A, 0, sizeof(A));
  if (form == 1) {
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) A.a[i][j] = 2.0 * W[i][j];
  } else {
    for (int col = 0; col < s; ++col) {
      int pv = col;
      for (int q = col + 1; q < s; ++q)
        if (std::fabs(W[q][col]) > std::fabs(W[pv][col])) pv = q;
      for (int j = 0; j < 2 * s; ++j) std::swap(W[col][j], W[pv][j]);
      const double inv = 1.0 / W[col][col];
      for (int j = 0; j < 2 * s; ++j) W[col][j] *= inv;
      for (int q = 0; q < s; ++q)
        if (q != col) {
          const double f = W[q][col];
          for (int j = 0; j < 2 * s; ++j) W[q][j] -= f * W[col][j];
        }
    }
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) A.a[i][j] = 0.5 * W[i][s + j];
  }
  const double* dU = U;
  const double* du = uprev;
  double* dR = R;
  if (kind == STDG_HOST) {
    CK(c, cudaMemcpyAsync(c->X1, U, c->slab_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->Xs, uprev, c->state_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
    dU = c->X1;
    du = c->Xs;
    dR = c->R;
  }
  // F(U) at every temporal node into X2, then the stage combination
  CKS(op_residual(c, dU, du, nullptr, c->X2));
  PK(c, 3, lodg_combine(dR, dU, c->X2, du, A, c->d.dt, form, c->nelem, c->s, c->nd * c->r, c->st));
  if (kind == STDG_HOST) {
    CK(c, cudaMemcpyAsync(R, dR, c->slab_len * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return STDG_OK;
}

stdg_status stdg_precond_apply(stdg_ctx* c, const double* U, const double* v, double* z, int kind) {
  if (!c || !U || !v || !z || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  if (!c->Pinv64) CKS(alloc(c, &c->Pinv64, (size_t)c->nelem * c->nd * c->s * c->s));
  const double* dU = U;
  const double* dv = v;
  double* dz = z;
  if (kind == STDG_HOST) {
    CK(c, cudaMemcpyAsync(c->X1, U, c->slab_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemcpyAsync(c->X2, v, c->slab_len * sizeof(double), cudaMemcpyHostToDevice, c->st));
    dU = c->X1;
    dv = c->X2;
    dz = c->R;
  }
  PK(c, 4, (pb_build<double>(c->dim, c->d.equation, c->a64, dU, c->Pinv64, c->st)));
  PK(c, 4, (pb_apply<double, double, double>(dz, dv, 1.0, c->Pinv64, 0, c->nelem, c->s, c->nd, c->r, c->st)));
  if (kind == STDG_HOST) {
    CK(c, cudaMemcpyAsync(z, dz, c->slab_len * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
  }
  return STDG_OK;
}

stdg_status stdg_profile_enable(stdg_ctx* c, int on) {
  if (!c) return STDG_ERR_INVALID_ARG;
  c->prof = on != 0;
  return STDG_OK;
}

stdg_status stdg_profile_read(stdg_ctx* c, stdg_profile* out, int reset) {
  if (!c || !out) return STDG_ERR_INVALID_ARG;
  DevGuard g(c->device);
  CK(c, cudaStreamSynchronize(c->st));
  prof_collect(c);
  for (int i = 0; i < kProfClasses; ++i) {
    out->launches[i] = c->prof_launches[i];
    out->ms[i] = c->prof_ms[i];
    if (reset) {
      c->prof_launches[i] = 0;
      c->prof_ms[i] = 0.0;
    }
  }
  return STDG_OK;
}

const char* stdg_last_error(const stdg_ctx* c) { return c ? c->err.c_str() : "null context"; }

const char* stdg_status_string(stdg_status st) {
  switch (st) {
    case STDG_OK: return "ok";
    case STDG_ERR_INVALID_ARG: return "invalid argument";
    case STDG_ERR_OOM: return "out of device memory";
    case STDG_ERR_CUDA: return "CUDA error";
    case STDG_ERR_NOT_CONVERGED: return "Newton did not converge";
    case STDG_ERR_GMRES_BREAKDOWN: return "GMRES breakdown";
    case STDG_ERR_NAN: return "non-finite residual";
    case STDG_ERR_TIMEOUT: return "timeout";
    case STDG_ERR_CANCELLED: return "cancelled";
    case STDG_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* stdg_version(void) { return "stdg-gb300 0.1"; }

stdg_status stdg_lgl_constants(int n, double* x, double* w, double* D) {
  if (!x || !w || !D || n < 2 || n > 16) return STDG_ERR_INVALID_ARG;
  lgl_rule(n, x, w);
  diff_matrix(n, x, D);
  return STDG_OK;
}

stdg_status stdg_predictor_matrix(int s, double* E) {
  if (!E || s < 2 || s > 5) return STDG_ERR_INVALID_ARG;
  lagrange_shift_matrix(s, 2.0, E);
  return STDG_OK;
}

}  // extern "C"
