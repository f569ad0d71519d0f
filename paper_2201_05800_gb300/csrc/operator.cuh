// Fused space-time DG-SEM operator: residual R(U), or J(U) v, of one time slab.
//
// One CTA owns `epb` consecutive elements and walks the s temporal nodes of
// their slab.  For every temporal node m:
//   0. thread per node: stage the element tiles of node m in shared memory
//      (coalesced loads, component-planar, node stride padded to an odd count):
//      U (residual), U + eps v (finite-difference Jv) or U and v (exact Jv), and
//      evaluate f_a(u) and the wave speed |v_a| + c for all directions a from the
//      staged values (one reciprocal of rho, one pressure, one sound speed)
//   1. (viscous term only) gradients of the staged lines
//   2. thread per node: volume term  -sum_a (2/h_a) (D f_a)      -> smem acc
//   3. thread per face point, one direction a at a time: Rusanov flux and the
//      strong-form face correction -(2/h_a)(1/w_end)(H.n - f_a(u).n).  A face
//      between two elements of the CTA is computed once and applied to both
//      sides from shared memory; for the others the neighbour trace is read
//      from global memory (L2) and its flux and wave speed evaluated.
//   4. thread per output value (coalesced): temporal coupling
//        R_m = sum_j omega_j Dtau[j][m] U_j + [m=0] u_prev - [m=s-1] U_s
//              + dt/2 omega_m F_m
//      (Eq. DG_in_time moved to one side so that dR/dU is Eq. Jacobian_ST),
//      with U_j (or v_j) read from global memory (L2).
// Strong form of the spatial operator (Sec. 3.1 with the SBP property of
// Eq. SBP): F_I = -sum_a (2/h_a) [ sum_j D[i_a][j] f_a(u_(I,i_a->j))
//      + (1/w_N) [i_a = N] (H_a^+ - f_a(u_I)) - (1/w_0) [i_a = 0] (H_a^- - f_a(u_I)) ].
// Only one temporal node is staged at a time so that many elements are
// resident per SM (the whole bench grid fits one wave).  The kernel is
// FP64-pipe bound in FP64 (ncu), so FP64 operations are avoided where
// possible: 2/h_a is folded into D, 1/eps and the GMRES left scaling 1/omega_m
// into the output factors, wave speeds are computed once per node, shared
// faces once per face.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace stdg {

// Pointwise state that the spatial operator sees in each mode.
template <int MODE, class T>
__device__ __forceinline__ auto eval_state(T u, T v, T eps) {
  if constexpr (MODE == kModeJvExact) return Dual<T>{u, v};
  else if constexpr (MODE == kModeJvFD) return u + eps * v;
  else return u;
}
// State of a staged tile node (the FD tile already holds U + eps v).
template <int MODE, class T>
__device__ __forceinline__ auto tile_state(T u, T v) {
  if constexpr (MODE == kModeJvExact) return Dual<T>{u, v};
  else return u;
}
template <class T> __device__ __forceinline__ T tangent(Dual<T> x) { return x.d; }
template <class T> __device__ __forceinline__ T tangent(T x) { return T(0); }


// Shared-memory footprint (bytes) of one CTA.
template <int DIM, int R, class T, int MODE>
__host__ __device__ inline size_t op_smem_bytes(int n, int s, int epb) {
  (void)s;
  int nd = 1;
  for (int a = 0; a < DIM; ++a) nd *= n;
  int ndp = nd | 1;
  size_t vbytes = (MODE == kModeJvExact) ? 2 * sizeof(T) : sizeof(T);
  size_t b = (size_t)epb * R * ndp * sizeof(T);                     // state tile of node m
  if (MODE == kModeJvExact) b += (size_t)epb * R * ndp * sizeof(T);  // direction tile of node m
  b += (size_t)epb * DIM * R * ndp * vbytes;                        // fluxes
  b += (size_t)epb * R * ndp * vbytes;                              // accumulators
  b += (size_t)epb * DIM * ndp * vbytes;                            // wave speeds
  b += (3 * kMaxN * kMaxN + kMaxS * kMaxS) * sizeof(T);             // scaled D per direction, C
  if (R == 1) {                                                     // viscous term (scalar equations)
    b += (size_t)epb * DIM * ndp * vbytes;                          // gradients
    b += (size_t)epb * DIM * 2 * (nd / n) * vbytes;                 // face jumps
  }
  b += (size_t)epb * DIM * 2 * sizeof(int);                         // neighbour elements
  return b;
}

// One CTA's work: elements [tile * epb, tile * epb + epb) of the slab described
// by k, with the CTA's dynamic shared memory.  NPX/NTX: compile-time n and s
// when FIXED, else upper bounds (runtime n, s).  Ends with a __syncthreads, so
// a CTA may call it again for another tile.
template <int DIM, int EQ, class T, int MODE, int NPX, int NTX, bool FIXED>
__device__ __forceinline__ void st_operator_tile(const OpArgs<T>& k, long long tile, unsigned char* smem_raw,
                                                 double* sums = nullptr, int m_first = 0, int m_step = 1) {
  using P = Phys<EQ, DIM>;
  constexpr int R = P::R;
  using V = typename std::conditional<MODE == kModeJvExact, Dual<T>, T>::type;

  const int n = FIXED ? NPX : k.n;
  const int s = FIXED ? NTX : k.s;
  const int nd = FIXED ? ipow_c(NPX, DIM) : k.nd;
  const int ndp = nd | 1;
  const int nf = nd / n;  // nodes on one face
  const int epb = k.epb;

  const long long e0 = tile * epb;
  const int nel = (int)((k.nelem - e0) < epb ? (k.nelem - e0) : epb);
  const int tid = threadIdx.x, nth = blockDim.x;

  T* su = reinterpret_cast<T*>(smem_raw);                             // [epb][R][ndp] state of node m
  T* sv = su + (size_t)epb * R * ndp;                                  // [epb][R][ndp] direction (exact)
  V* sf = reinterpret_cast<V*>(MODE == kModeJvExact ? sv + (size_t)epb * R * ndp : sv);  // [epb][DIM][R][ndp]
  V* sr = sf + (size_t)epb * DIM * R * ndp;                            // [epb][R][ndp]
  V* sl = sr + (size_t)epb * R * ndp;                                  // [epb][DIM][ndp] wave speeds
  T* sD = reinterpret_cast<T*>(sl + (size_t)epb * DIM * ndp);          // [3][kMaxN][kMaxN]  (2/h_a) D
  T* sC = sD + 3 * kMaxN * kMaxN;                                      // [kMaxS][kMaxS]  C
  V* sq = reinterpret_cast<V*>(sC + kMaxS * kMaxS);                    // [epb][DIM][ndp] gradients (R == 1)
  V* sjm = sq + (size_t)epb * DIM * ndp;                               // [epb][DIM][2][nf] face jumps (R == 1)
  int* snb = reinterpret_cast<int*>(R == 1 ? sjm + (size_t)epb * DIM * 2 * nf : sq);  // [epb][DIM][2]
  const bool visc = (R == 1) && k.nu != T(0);
  // index helpers: divisions by n, n^2, n^d are by constants (FIXED) or by multiply-high
  auto div_n = [&](int t) { return FIXED ? t / NPX : fast_div(t, k.mg_n); };
  auto div_n2 = [&](int t) { return FIXED ? t / (NPX * NPX) : fast_div(t, k.mg_n2); };
  auto div_nd = [&](int t) { return FIXED ? t / ipow_c(NPX, DIM) : fast_div(t, k.mg_nd); };
  auto div_nf = [&](int t) { return DIM == 1 ? t : (DIM == 2 ? div_n(t) : div_n2(t)); };
  auto div_stride = [&](int t, int a) { return a == 0 ? t : (a == 1 ? div_n(t) : div_n2(t)); };
  for (int i = tid; i < 3 * kMaxN * kMaxN; i += nth) {
    const int a = i / (kMaxN * kMaxN), q = i % (kMaxN * kMaxN);
    sD[i] = k.ginv[a] * k.D[q / kMaxN][q % kMaxN];
  }
  for (int i = tid; i < kMaxS * kMaxS; i += nth) sC[i] = k.C[i / kMaxS][i % kMaxS];
  // periodic neighbour elements of the tile, [el][a][side] (side 1: +e_a), 32-bit arithmetic
  for (int i = tid; i < nel * DIM * 2; i += nth) {
    const int side = i & 1, a = (i >> 1) % DIM, el = (i >> 1) / DIM;
    const unsigned e = (unsigned)(e0 + el);
    const unsigned K0 = (unsigned)k.K[0], K1 = (unsigned)k.K[1];
    int ec[3] = {(int)(e % K0), (int)((e / K0) % K1), (int)(e / (K0 * K1))};
    ec[a] += side ? 1 : -1;
    if (ec[a] < 0) ec[a] += k.K[a];
    if (ec[a] >= k.K[a]) ec[a] -= k.K[a];
    snb[i] = (ec[2] * k.K[1] + ec[1]) * k.K[0] + ec[0];
  }

  const size_t tnode = (size_t)nd * R;  // values of one element at one temporal node
  const T ev = k.eps * k.vscale;         // FD Jv: U + (eps vscale) v, one FMA per value
  const int strides[3] = {1, n, n * n};
  // the tile the temporal coupling acts on: U for the residual, v for J v
  const T* gtile = (MODE == kModeResidual) ? k.U : k.v;

  // each temporal node is self-contained: F at node m and the linear temporal coupling read
  // from global memory, so a CTA may take any subset of them
  for (int m = m_first; m < s; m += m_step) {
    // ---- 0. stage node m of the CTA's elements (coalesced global reads) and evaluate the
    //         fluxes f_a(u) and wave speeds |v_a| + c at every node: each thread works on the
    //         node it staged (one reciprocal of rho, one pressure, one sound speed per node)
    for (int t = tid; t < nel * nd; t += nth) {
      const int el = div_nd(t), node = t - el * nd;
      const size_t g0 = ((size_t)(e0 + el) * s + m) * tnode + (size_t)node * R;
      const size_t so0 = ((size_t)el * R) * ndp + node;
      V u[R];
#pragma unroll
      for (int c = 0; c < R; ++c) {
        const size_t g = g0 + c, so = so0 + (size_t)c * ndp;
        if constexpr (MODE == kModeJvFD) {
          const T x = fma(ev, k.v[g], k.U[g]);
          su[so] = x;
          u[c] = x;
        } else if constexpr (MODE == kModeJvExact) {
          const T x = k.U[g], y = k.vscale * k.v[g];
          su[so] = x;
          sv[so] = y;
          u[c] = tile_state<MODE>(x, y);
        } else {
          const T x = k.U[g];
          su[so] = x;
          u[c] = tile_state<MODE>(x, T(0));
          if (sums) sums[1] = fma((double)x, (double)x, sums[1]);
        }
      }
      V f[DIM][R];
      V lam[DIM];
      P::flux_all_speed(u, f, lam, k);
      V* sfe = sf + (size_t)el * DIM * R * ndp;
      V* sle = sl + (size_t)el * DIM * ndp;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        sle[a * ndp + node] = lam[a];
#pragma unroll
        for (int c = 0; c < R; ++c) sfe[(a * R + c) * ndp + node] = f[a][c];
      }
    }
    __syncthreads();
    // ---- 1. (viscous term) gradients along every direction from the staged lines
    if constexpr (R == 1) {
      if (visc) {
        for (int t = tid; t < nel * nd; t += nth) {
          const int el = div_nd(t), node = t - el * nd;
          // gradient along each direction: (2/h_a) sum_j D[i_a][j] u along the line
          const int q1 = div_n(node), q2 = div_n(q1);
          const int idx[3] = {node - q1 * n, q1 - q2 * n, q2};
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            const int base = node - idx[a] * strides[a];
            const T* Da = sD + (a * kMaxN + idx[a]) * kMaxN;
            V q = Lift<V, T>::from(T(0));
#pragma unroll
            for (int j = 0; j < NPX; ++j) {
              if (FIXED || j < n) {
                const size_t sj = ((size_t)el * R) * ndp + base + j * strides[a];
                q = q + Da[j] * tile_state<MODE>(su[sj], MODE == kModeJvExact ? sv[sj] : T(0));
              }
            }
            sq[((size_t)el * DIM + a) * ndp + node] = q;
          }
        }
        __syncthreads();
      }
    }
    // ---- 2. volume term
    for (int t = tid; t < nel * nd; t += nth) {
      const int el = div_nd(t), node = t - el * nd;
      const int q1 = div_n(node), q2 = div_n(q1);
      const int idx[3] = {node - q1 * n, q1 - q2 * n, q2};
      const V* sfe = sf + (size_t)el * DIM * R * ndp;
      V acc[R];
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] = Lift<V, T>::from(T(0));
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int ia = idx[a];
        const int base = node - ia * strides[a];
        const T* Da = sD + (a * kMaxN + ia) * kMaxN;
#pragma unroll
        for (int c = 0; c < R; ++c) {
#pragma unroll
          for (int j = 0; j < NPX; ++j) {
            if (FIXED || j < n) acc[c] = acc[c] - Da[j] * sfe[(a * R + c) * ndp + base + j * strides[a]];
          }
        }
      }
      if constexpr (R == 1) {
        if (visc) {
          // -nu sum_a (2/h_a) (1/w_i) sum_k w_k D[k][i] q_a(k)   (SIPG volume term)
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            const int ia = idx[a];
            const int base = node - ia * strides[a];
            const V* sqa = sq + ((size_t)el * DIM + a) * ndp;
#pragma unroll
            for (int j = 0; j < NPX; ++j)
              if (FIXED || j < n) acc[0] = acc[0] - k.vDW[a][ia][j] * sqa[base + j * strides[a]];
          }
        }
      }
      V* sre = sr + (size_t)el * R * ndp;
#pragma unroll
      for (int c = 0; c < R; ++c) sre[c * ndp + node] = acc[c];
    }
    __syncthreads();
    // ---- 3. face corrections, one direction at a time.  Items [0, nel*nf) are the
    //         upper faces (+e_a) of the CTA's elements: a face whose neighbour is
    //         also in this CTA is computed once and applied to both sides from
    //         shared memory.  Items [nel*nf, 2*nel*nf) are the lower faces whose
    //         neighbour lies outside the CTA (the others were done by the
    //         neighbour's upper item).  Within a direction no two items touch the
    //         same node (n >= 2).
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const T g = k.ginv[a] * k.winv_end;
      const T gh = T(0.5) * g;
      for (int t = tid; t < 2 * nel * nf; t += nth) {
        const int side = t < nel * nf ? 1 : 0;  // 1: upper face (normal +e_a), 0: lower face
        const int tt = side ? t : t - nel * nf;
        const int el = div_nf(tt);
        const int fidx = tt - el * nf;
        // own node: insert i_a into the face index
        const int hi = div_stride(fidx, a);
        const int lo = fidx - hi * strides[a];
        const int ia_own = side ? n - 1 : 0;
        const int own = lo + ia_own * strides[a] + hi * strides[a] * n;
        const int nbr_node = lo + (n - 1 - ia_own) * strides[a] + hi * strides[a] * n;
        // neighbour element (periodic), from the tile's table
        const long long en = snb[(el * DIM + a) * 2 + side];
        const long long eln = en - e0;
        const bool internal = eln >= 0 && eln < nel;
        if (!side && internal) continue;  // computed by the neighbour's upper item
        const size_t so = ((size_t)el * R) * ndp + own;
        const V* sfe = sf + (size_t)el * DIM * R * ndp;
        V um[R], up[R], fm[R], fp[R];
        V qm = Lift<V, T>::from(T(0)), qp = Lift<V, T>::from(T(0));  // normal gradients (viscous)
#pragma unroll
        for (int c = 0; c < R; ++c) {
          fm[c] = sfe[(a * R + c) * ndp + own];
          um[c] = tile_state<MODE>(su[so + c * ndp], MODE == kModeJvExact ? sv[so + c * ndp] : T(0));
        }
        const V lm = sl[((size_t)el * DIM + a) * ndp + own];
        V lp;
        if (internal) {
          const size_t son = ((size_t)eln * R) * ndp + nbr_node;
          const V* sfn = sf + (size_t)eln * DIM * R * ndp;
#pragma unroll
          for (int c = 0; c < R; ++c) {
            fp[c] = sfn[(a * R + c) * ndp + nbr_node];
            up[c] = tile_state<MODE>(su[son + c * ndp], MODE == kModeJvExact ? sv[son + c * ndp] : T(0));
          }
          lp = sl[((size_t)eln * DIM + a) * ndp + nbr_node];
          if constexpr (R == 1)
            if (visc) qp = sq[((size_t)eln * DIM + a) * ndp + nbr_node];
        } else {
          const size_t gofs = ((size_t)en * s + m) * tnode + (size_t)nbr_node * R;
#pragma unroll
          for (int c = 0; c < R; ++c) {
            if constexpr (MODE == kModeJvFD) up[c] = fma(ev, k.v[gofs + c], k.U[gofs + c]);
            else up[c] = eval_state<MODE>(k.U[gofs + c], MODE == kModeResidual ? T(0) : k.vscale * k.v[gofs + c],
                                          k.eps);
          }
          lp = P::flux_speed(up, a, fp, k);
          if constexpr (R == 1) {
            if (visc) {
              // the neighbour's gradient at its face node from its line along e_a
              const int ib = n - 1 - ia_own;
              const T* Db = sD + (a * kMaxN + ib) * kMaxN;
              const size_t lbase = ((size_t)en * s + m) * tnode + (size_t)(lo + hi * strides[a] * n) * R;
#pragma unroll
              for (int j = 0; j < NPX; ++j) {
                if (FIXED || j < n) {
                  const size_t gj = lbase + (size_t)j * strides[a] * R;
                  if constexpr (MODE == kModeJvFD) qp = qp + Db[j] * fma(ev, k.v[gj], k.U[gj]);
                  else
                    qp = qp + Db[j] * eval_state<MODE>(k.U[gj], MODE == kModeResidual ? T(0) : k.vscale * k.v[gj],
                                                       k.eps);
                }
              }
            }
          }
        }
        if constexpr (R == 1)
          if (visc) qm = sq[((size_t)el * DIM + a) * ndp + own];
        V* sre = sr + (size_t)el * R * ndp;
        if (side) {  // own element below the face: uL = u-, uR = u+
          const V lam = dmax(lm, lp);
          V* srn = sr + (size_t)(internal ? eln : el) * R * ndp;
          // with H = (fm + fp)/2 - lam (up - um)/2:  H - fm = (df - lam du)/2 and
          // H - fp = -(df + lam du)/2, df = fp - fm, du = up - um
#pragma unroll
          for (int c = 0; c < R; ++c) {
            const V du = up[c] - um[c], df = fp[c] - fm[c];
            sre[c * ndp + own] = sre[c * ndp + own] - gh * (df - lam * du);  // n = +e_a
            if (internal) srn[c * ndp + nbr_node] = srn[c * ndp + nbr_node] - gh * (df + lam * du);  // n = -e_a
          }
          if constexpr (R == 1) {
            if (visc) {
              // jump [[u]] = uL - uR, average of nu grad u; the element below gets
              // -(2/h)(1/w_N)(-nu {q} + sigma [[u]]), the element above -(2/h)(1/w_0)(nu {q} - sigma [[u]])
              const V jmp = um[0] - up[0];
              const V avg = T(0.5) * (qm + qp);
              const V fb = k.nu * avg - k.pen[a] * jmp;
              sre[own] = sre[own] + g * fb;
              sjm[(((size_t)el * DIM + a) * 2 + 1) * nf + fidx] = jmp;
              if (internal) {
                srn[nbr_node] = srn[nbr_node] - g * fb;
                sjm[(((size_t)eln * DIM + a) * 2 + 0) * nf + fidx] = jmp;
              }
            }
          }
        } else {     // own element above the face: uL = u+, uR = u-
          const V lam = dmax(lp, lm);
          // own element above: H = (fp + fm)/2 - lam (um - up)/2, H - fm = (df - lam du)/2
          // with df = fp - fm, du = um - up
#pragma unroll
          for (int c = 0; c < R; ++c) {
            const V du = um[c] - up[c], df = fp[c] - fm[c];
            sre[c * ndp + own] = sre[c * ndp + own] + gh * (df - lam * du);
          }
          if constexpr (R == 1) {
            if (visc) {
              const V jmp = up[0] - um[0];
              const V avg = T(0.5) * (qp + qm);
              sre[own] = sre[own] - g * (k.nu * avg - k.pen[a] * jmp);
              sjm[(((size_t)el * DIM + a) * 2 + 0) * nf + fidx] = jmp;
            }
          }
        }
      }
      __syncthreads();
    }
    if constexpr (R == 1) {
      if (visc) {
        // ---- 3b. lift of the face jumps along the normal lines (symmetry term of the
        //          SIPG form): F_I += nu/2 (2/h_a)^2 (1/w_i) (D[N][i] [[u]]_up + D[0][i] [[u]]_lo)
        for (int t = tid; t < nel * nd; t += nth) {
          const int el = div_nd(t), node = t - el * nd;
          const int q1 = div_n(node), q2 = div_n(q1);
          const int idx[3] = {node - q1 * n, q1 - q2 * n, q2};
          V acc = sr[(size_t)el * ndp + node];
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            const int ia = idx[a];
            // face index: node with digit a removed
            const int lo = a == 0 ? 0 : (a == 1 ? idx[0] : idx[0] + idx[1] * n);
            const int hi = a == 0 ? idx[1] + idx[2] * n : (a == 1 ? idx[2] : 0);
            const int fidx = lo + hi * strides[a];
            const V* sja = sjm + ((size_t)el * DIM + a) * 2 * nf;
            acc = acc + k.vup[a][ia] * sja[nf + fidx] + k.vlo[a][ia] * sja[fidx];
          }
          sr[(size_t)el * ndp + node] = acc;
        }
        __syncthreads();
      }
    }
    // ---- 4. temporal coupling and output (coalesced: consecutive threads read and
    //         write consecutive values of the element's [node][c] block)
    //         out = sum_j cm_j x_j - [m = s-1] ce x_m + cfac * (spatial term), with the
    //         direction scale, the GMRES left scaling 1/omega_m and 1/eps folded in.
    {
      const bool ls = MODE != kModeResidual && k.lscale;
      const T sm = ls ? k.inv_omega[m] : T(1);
      const T vs = MODE == kModeResidual ? T(1) : k.vscale;
      const T hw = ls ? k.half_dt : k.half_dt * k.omega[m];
      const T cfac = MODE == kModeJvFD ? hw * k.inv_eps : hw;
      T cm[NTX];
#pragma unroll
      for (int j = 0; j < NTX; ++j) cm[j] = (FIXED || j < s) ? (sm * vs) * sC[j * kMaxS + m] : T(0);
      const T ce = sm * vs;
      for (int t = tid; t < nel * (int)tnode; t += nth) {
        const int c = t % R;
        const int r2 = t / R;
        const int el = div_nd(r2);
        const int node = r2 - el * nd;
        const size_t gb = (size_t)(e0 + el) * s * tnode + (size_t)node * R + c;  // (e, j = 0, node, c)
        const size_t g = gb + (size_t)m * tnode;
        const V Fv = sr[((size_t)el * R + c) * ndp + node];
        T lin = T(0);
#pragma unroll
        for (int j = 0; j < NTX; ++j)
          if (FIXED || j < s) lin += cm[j] * gtile[gb + (size_t)j * tnode];
        if (m == s - 1) lin -= ce * gtile[g];
        if (MODE == kModeResidual) {
          // u_prev is only read when R is written (F-only launches pass no u_prev)
          if (k.out) {
            if (m == 0) lin += k.uprev[(size_t)(e0 + el) * tnode + (size_t)node * R + c];
            const T rv = lin + cfac * val(Fv);
            k.out[g] = rv;
            if (sums) {
              const double wv = k.v0w ? (double)rv * (double)k.inv_omega[m] : (double)rv;
              sums[0] = fma((double)rv, (double)rv, sums[0]);
              sums[2] = fma(wv, wv, sums[2]);
              if (k.v0d) k.v0d[g] = wv;
              if (k.v0f) k.v0f[g] = (float)wv;
            }
          }
          if (k.fout) k.fout[g] = val(Fv);
        } else if (MODE == kModeJvFD) {
          k.out[g] = fma(cfac, val(Fv) - k.F0[g], lin);
        } else {
          k.out[g] = fma(cfac, tangent(Fv), lin);
        }
      }
    }
    __syncthreads();
  }
}

template <int DIM, int EQ, class T, int MODE, int NPX, int NTX, bool FIXED>
__global__ void __launch_bounds__(256) st_operator_kernel(const __grid_constant__ OpArgs<T> k) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ms = k.msplit > 1 ? k.msplit : 1;
  const long long tile = blockIdx.x / ms;
  const int m_first = blockIdx.x % ms;
  if (MODE == kModeResidual && k.nrm && k.out) {
    // residual with its norms: per-thread sums, then a fixed-order block sum
    double sums[3] = {0.0, 0.0, 0.0};
    st_operator_tile<DIM, EQ, T, MODE, NPX, NTX, FIXED>(k, tile, smem_raw, sums, m_first, ms);
    __shared__ double red[256 / 32][3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double v = sums[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
      k.nrm[(size_t)blockIdx.x * k.nrm_stride + threadIdx.x] = v;
    }
  } else {
    st_operator_tile<DIM, EQ, T, MODE, NPX, NTX, FIXED>(k, tile, smem_raw, nullptr, m_first, ms);
  }
}

}  // namespace stdg
