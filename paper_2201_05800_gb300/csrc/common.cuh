// Device-side building blocks of the space-time DG-SEM operator: kernel
// arguments, dual numbers (forward-mode derivatives for the exact Jacobian-
// vector product) and the convective physics with the Rusanov flux.
//
// Physics (arXiv:2201.05800):
//   Euler equations, Eqs. eulereq/defu and the flux f_i printed after them
//   (Sec. 7.3); linear advection f_i = a_i u; Burgers f_i = u^2/2.
//   Rusanov flux, Eq. flux:llf, on a face with normal +e_a between a left state
//   uL and a right state uR:  H = (f_a(uL) + f_a(uR))/2 - lambda/2 (uR - uL),
//   lambda = max(|v_a| + c) over the two states (ties take the left state).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "stdg.h"

namespace stdg {

constexpr int kMaxN = 8;  // LGL nodes per direction (spatial degree N <= 7)
constexpr int kMaxS = 5;  // temporal LGL nodes N_tau

// Operator modes.
enum OpMode {
  kModeResidual = 0,  // out = R(U; u_prev) (if out), fout = F(U) (if fout)
  kModeJvFD = 1,      // out = J(U) v by a one-sided difference of F around F0 = F(U)
  kModeJvExact = 2    // out = J(U) v by forward-mode (dual-number) differentiation
};

// Arguments of one operator launch.  Constants are already scaled for the
// strong form: F_I = -sum_a ginv_a [ (D f_a)_I + winv_end (face corrections) ].
template <class T>
struct OpArgs {
  int n, s, nd, epb;       // LGL nodes per direction, temporal nodes, n^d, elements per block
  int K[3];                // elements per direction
  long long nelem;
  T D[kMaxN][kMaxN];       // D[i][j] = l_j'(xi_i) on [-1, 1]
  T C[kMaxS][kMaxS];       // C[j][m] = omega_j Dtau[j][m], i.e. (D_tau^T M_tau)[m][j]
  T omega[kMaxS];          // temporal LGL weights
  T ginv[3];               // 2 / h_a
  T winv_end;              // 1 / w_0 = 1 / w_N (end weights of the spatial LGL rule)
  T half_dt;               // Delta t / 2
  T gamma;
  T adv[3];
  T eps;                   // FD step (kModeJvFD)
  T inv_eps;               // 1 / eps
  T vscale;                // v is read as vscale * v (kModeJvFD / kModeJvExact)
  int lscale;              // Jv modes: rows of temporal node m divided by omega_m
  T inv_omega[kMaxS];      // 1 / omega_m
  // symmetric interior penalty viscous term (scalar equations, nu > 0):
  T nu;                    // viscosity (0: inviscid)
  T pen[3];                // penalty sigma_a = nu eta / h_a
  T vDW[3][kMaxN][kMaxN];  // nu (2/h_a) (w_k / w_i) D[k][i]: volume term, [a][i][k]
  T vup[3][kMaxN];         // nu/2 (2/h_a)^2 D[N][i] / w_i: lift of the upper-face jump
  T vlo[3][kMaxN];         // nu/2 (2/h_a)^2 D[0][i] / w_i: lift of the lower-face jump
  T vdiag[3][kMaxN];       // diagonal of the viscous term of F per direction (preconditioner)
  // multipliers for division by n, n^2 and n^d (fast_div; 0 for a divisor of 1)
  unsigned mg_n, mg_n2, mg_nd;
  const T* U;              // slab, [e][m][node][c]
  const T* v;              // direction, same layout
  const T* F0;             // F(U), same layout (kModeJvFD)
  const T* uprev;          // previous slab trace, [e][node][c] (kModeResidual)
  T* out;                  // R or Jv (may be null in kModeResidual)
  T* fout;                 // F(U) (kModeResidual, may be null)
  // kModeResidual with out set, optional: per-block sums |R|^2, |U|^2 and |W^-1 R|^2 at
  // nrm[block * nrm_stride + 0..2] (W = M_tau if v0w, else I), and W^-1 R written to v0d
  // (FP64) or v0f (FP32): the Newton norms and the first Krylov vector in the same pass
  double* nrm;
  int nrm_stride, v0w;
  // temporal nodes split over CTAs: CTA b works on element tile b / msplit and on the
  // temporal nodes m = b % msplit, b % msplit + msplit, ... (0 or 1: one CTA per tile)
  int msplit;
  // jv_tangent_kernel: tile distance of the L2 prefetch (the CTAs resident at once), 0 = none
  int prefetch;
  double* v0d;
  float* v0f;
  // error word of kernels with bounded waits (bit 0: a wait gave up), or null
  unsigned* err;
};

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

// Division of a small index by a runtime divisor d without an integer divide:
// q = floor(t * ceil(2^32 / d) / 2^32) is exact for t, d < 2^16 (the error term
// t (m d - 2^32) / 2^32 stays below 1).  mg = 0 encodes d = 1.
__host__ __device__ inline unsigned fast_div_magic(unsigned d) {
  return d <= 1 ? 0u : (unsigned)(((1ull << 32) + d - 1) / d);
}
__device__ __forceinline__ int fast_div(int t, unsigned mg) { return mg ? (int)__umulhi((unsigned)t, mg) : t; }

// ---------------------------------------------------------------- dual numbers
template <class T>
struct Dual {
  T v, d;
};

template <class T> __device__ __forceinline__ T val(T x) { return x; }
template <class T> __device__ __forceinline__ T val(Dual<T> x) { return x.v; }

template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return {a.v - b, a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return {a - b.v, -b.d}; }
template <class T> __device__ __forceinline__ Dual<T> recip(Dual<T> a) {
  T r = T(1) / a.v;
  return {r, -a.d * r * r};
}
template <class T> __device__ __forceinline__ T recip(T a) { return T(1) / a; }
template <class T> __device__ __forceinline__ Dual<T> dsqrt(Dual<T> a) {
  T r = sqrt(a.v);
  return {r, a.d * (T(0.5) / r)};
}
template <class T> __device__ __forceinline__ T dsqrt(T a) { return sqrt(a); }
template <class T> __device__ __forceinline__ Dual<T> dabs(Dual<T> a) { return a.v >= T(0) ? a : -a; }
template <class T> __device__ __forceinline__ T dabs(T a) { return fabs(a); }
// max with the branch chosen on the values; ties take the first argument
template <class V> __device__ __forceinline__ V dmax(V a, V b) { return val(a) >= val(b) ? a : b; }

template <class V, class T> struct Lift { __device__ static V from(T x) { return x; } };
template <class T> struct Lift<Dual<T>, T> { __device__ static Dual<T> from(T x) { return {x, T(0)}; } };

// ---------------------------------------------------------------- physics
template <int EQ, int DIM> struct Phys;

template <int DIM>
struct Phys<STDG_ADVECTION, DIM> {
  static constexpr int R = 1;
  template <class V, class T>
  __device__ static void flux_all(const V* u, V (*f)[R], const OpArgs<T>& k) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) f[a][0] = k.adv[a] * u[0];
  }
  template <class V, class T>
  __device__ static void flux(const V* u, int a, V* f, const OpArgs<T>& k) { f[0] = k.adv[a] * u[0]; }
  template <class V, class T>
  __device__ static V speed(const V* u, int a, const OpArgs<T>& k) { return Lift<V, T>::from(fabs(k.adv[a])); }
  template <class V, class T>
  __device__ static void flux_all_speed(const V* u, V (*f)[R], V* lam, const OpArgs<T>& k) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      f[a][0] = k.adv[a] * u[0];
      lam[a] = Lift<V, T>::from(fabs(k.adv[a]));
    }
  }
  template <class V, class T>
  __device__ static V flux_speed(const V* u, int a, V* f, const OpArgs<T>& k) {
    f[0] = k.adv[a] * u[0];
    return Lift<V, T>::from(fabs(k.adv[a]));
  }
};

template <int DIM>
struct Phys<STDG_BURGERS, DIM> {
  static constexpr int R = 1;
  template <class V, class T>
  __device__ static void flux_all(const V* u, V (*f)[R], const OpArgs<T>& k) {
    V h = T(0.5) * (u[0] * u[0]);
#pragma unroll
    for (int a = 0; a < DIM; ++a) f[a][0] = h;
  }
  template <class V, class T>
  __device__ static void flux(const V* u, int a, V* f, const OpArgs<T>& k) { f[0] = T(0.5) * (u[0] * u[0]); }
  template <class V, class T>
  __device__ static V speed(const V* u, int a, const OpArgs<T>& k) { return dabs(u[0]); }
  template <class V, class T>
  __device__ static void flux_all_speed(const V* u, V (*f)[R], V* lam, const OpArgs<T>& k) {
    V h = T(0.5) * (u[0] * u[0]);
    V l = dabs(u[0]);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      f[a][0] = h;
      lam[a] = l;
    }
  }
  template <class V, class T>
  __device__ static V flux_speed(const V* u, int a, V* f, const OpArgs<T>& k) {
    f[0] = T(0.5) * (u[0] * u[0]);
    return dabs(u[0]);
  }
};

template <int DIM>
struct Phys<STDG_EULER, DIM> {
  static constexpr int R = DIM + 2;
  // pressure p = (gamma - 1) (E - |m|^2 / (2 rho)) given 1/rho
  template <class V, class T>
  __device__ static V pressure(const V* u, V irho, const OpArgs<T>& k) {
    V m2 = u[1] * u[1];
#pragma unroll
    for (int b = 1; b < DIM; ++b) m2 = m2 + u[1 + b] * u[1 + b];
    return (k.gamma - T(1)) * (u[R - 1] - T(0.5) * (m2 * irho));
  }
  template <class V, class T>
  __device__ static void flux_all(const V* u, V (*f)[R], const OpArgs<T>& k) {
    V irho = recip(u[0]);
    V p = pressure(u, irho, k);
    V Ep = u[R - 1] + p;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      V va = u[1 + a] * irho;
      f[a][0] = u[1 + a];
#pragma unroll
      for (int b = 0; b < DIM; ++b) f[a][1 + b] = (b == a) ? u[1 + b] * va + p : u[1 + b] * va;
      f[a][R - 1] = Ep * va;
    }
  }
  template <class V, class T>
  __device__ static void flux(const V* u, int a, V* f, const OpArgs<T>& k) {
    V irho = recip(u[0]);
    V p = pressure(u, irho, k);
    V va = u[1 + a] * irho;
    f[0] = u[1 + a];
#pragma unroll
    for (int b = 0; b < DIM; ++b) f[1 + b] = (b == a) ? u[1 + b] * va + p : u[1 + b] * va;
    f[R - 1] = (u[R - 1] + p) * va;
  }
  // fluxes in every direction and the wave speeds |v_a| + c, sharing 1/rho, p and c
  template <class V, class T>
  __device__ static void flux_all_speed(const V* u, V (*f)[R], V* lam, const OpArgs<T>& k) {
    V irho = recip(u[0]);
    V p = pressure(u, irho, k);
    V Ep = u[R - 1] + p;
    V c = dsqrt(k.gamma * (p * irho));
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      V va = u[1 + a] * irho;
      f[a][0] = u[1 + a];
#pragma unroll
      for (int b = 0; b < DIM; ++b) f[a][1 + b] = (b == a) ? u[1 + b] * va + p : u[1 + b] * va;
      f[a][R - 1] = Ep * va;
      lam[a] = dabs(va) + c;
    }
  }
  // flux in direction a and the wave speed |v_a| + c
  template <class V, class T>
  __device__ static V flux_speed(const V* u, int a, V* f, const OpArgs<T>& k) {
    V irho = recip(u[0]);
    V p = pressure(u, irho, k);
    V va = u[1 + a] * irho;
    f[0] = u[1 + a];
#pragma unroll
    for (int b = 0; b < DIM; ++b) f[1 + b] = (b == a) ? u[1 + b] * va + p : u[1 + b] * va;
    f[R - 1] = (u[R - 1] + p) * va;
    return dabs(va) + dsqrt(k.gamma * (p * irho));
  }
  // |v_a| + sqrt(gamma p / rho)
  template <class V, class T>
  __device__ static V speed(const V* u, int a, const OpArgs<T>& k) {
    V irho = recip(u[0]);
    V p = pressure(u, irho, k);
    return dabs(u[1 + a] * irho) + dsqrt(k.gamma * (p * irho));
  }
};

}  // namespace stdg
