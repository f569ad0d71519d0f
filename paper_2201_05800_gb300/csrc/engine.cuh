// Batched, device-driven Newton-Krylov engine: many independent slab solves
// (slots) advance together, one state-machine step per "tick".
//
// Every slot solves its own slab system R(U) = 0 (Eq. DG_vs_RK:DG) by Newton
// (Sec. 6.3) with a right-preconditioned flexible GMRES(m) inner solve: the
// point-block preconditioner of precond.cuh, the Krylov basis V, the
// preconditioned directions Z = P^-1 V and the exact (forward-mode) FP32
// Jacobian-vector products; the Newton residual, the solution update and the
// Hessenberg/Givens arithmetic are FP64 (iterative refinement).  No restarts:
// a Newton step takes the GMRES iterate after at most m iterations.
//
// The whole solver state of a slot lives on the device: its vectors in one
// allocation of the engine's arena and its scalars (phase, Hessenberg matrix,
// rotations, coefficients) in a SlotCtl record.  A tick is a fixed sequence of
// launches over all slots, each kernel walking a list of work items
// (slot, tile) and skipping the slots whose phase does not need it:
//   1. build   P_I^-1 from U                       (slots in kPhResid)
//   2. op      R(U) in FP64                        (kPhResid)
//   3. op      w = J z_j in FP32                   (kPhArnoldi)
//   4. dot     |R|^2, or V_i . w for i <= j + 1    (kPhResid, kPhArnoldi, kPhReorth)
//   5. control one warp per slot: sums its partials in a fixed order, then
//              Newton test / Hessenberg column / Givens rotation / triangular
//              solve, and picks the next phase and this tick's update
//   6. update  w -= V c, z = P^-1 (w / |w|), U += Z y, u^{n+1} = U^s
// No host synchronisation inside a tick; slots are independent (no reduction
// crosses slots and every reduction has a fixed order), so a slot's result
// does not depend on which other slots share the launches.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace stdg {

constexpr int kEngMaxM = 31;  // Krylov dimension: basis of m + 1 <= 32 rows
constexpr int kEngRows = 32;
constexpr int kEngThreads = 256;
// The controller block of a slot with more than kCtlWideItems chunk items reduces its partial
// sums with kCtlWideWarps warps (else kEngThreads / 32); the choice depends on the slot alone.
constexpr int kCtlWideItems = 512, kCtlWideWarps = 32;
// Slots of at least kDotWideLen values take the dot pass with 16 rows per group.
constexpr size_t kDotWideLen = (size_t)1 << 21;

enum EngPhase { kPhIdle = 0, kPhResid = 1, kPhArnoldi = 2, kPhReorth = 3, kPhDone = 4 };
enum EngUpd { kUpdNone = 0, kUpdInit = 1, kUpdGS = 2, kUpdGSZ = 3, kUpdSolve = 4, kUpdExtract = 5 };

// Device pointers and sizes of one slot.
struct SlotBuf {
  double* U;      // Newton iterate, slab layout [e][m][node][c]
  double* R;      // Newton residual
  double* uprev;  // u^n on entry, u^{n+1} after the solve, [e][node][c]
  float* U32;     // FP32 copy of U (base point of the Jacobian-vector products)
  float* Pinv;    // P_I^-1 per spatial node, [e][m][j][node]
  float* V;       // Krylov basis, m + 1 rows of L values (unnormalised, v_i = sig_i V_i)
  float* Z;       // preconditioned directions z_i = P^-1 v_i, m rows
  long long nelem;
  int s, nd, r;
  int chunk_elems;  // elements per work item of the build / dot / update kernels
  size_t L;         // slab length nelem * s * nd * r
  int item0, nitems;  // this slot's work items in the chunk list (control reduction)
  int op0, nop;       // this slot's tiles in the operator item list (skipped together)
  int vec4;           // L % 4 == 0: every row starts on 16 bytes (vector loads in dot / update)
  int stride, offset; // the slot takes part in tick t when (t + offset) % stride == 0
  // element tensor-product preconditioner (scalar equations; kron = 1), see eng_kron_kernel:
  // kdat = [Vx^-1 | Vx | Vy^-1 | Vy] (n x n each) then P_k^-1 (s x s) per mode k of the element
  int kron, dim, n;
  int pbtm;  // Euler slots without STDG_PRECOND_POINT_BLOCK: z = diag(1 / omega_m) v (no block array)
  const float* kdat;
  // global fast-diagonalisation preconditioner (scalar slots on periodic grids whose element
  // counts are powers of two; fdm = 1 replaces kron), see engine_fdm.cu:
  // fdat = tw_x | F_x | B_x | lam_x | tw_y | F_y | B_y | lam_y (offsets below, in floats)
  int fdm, fkx, fky, fny, flogx, flogy;
  int f_twx, f_Fx, f_Bx, f_lx, f_twy, f_Fy, f_By, f_ly;
  const float* fdat;
  float2* fx;  // complex scratch of L values, [kx][jx][m][ey][iy]
};

// Scalar solver state of one slot (FP64).
struct SlotCtl {
  int phase, j, m, upd, upd_row, upd_k;
  int newton_its, gmres_its, resid_evals, jv_evals, newton_maxit, status;
  double rtol, atol, gmres_rtol;
  double res0, target, res, beta, tol, zscale;
  double coef[kEngRows];
  double sig[kEngRows + 1];
  double g[kEngRows + 1];
  double cs[kEngRows], sn[kEngRows];
  double H[kEngRows * kEngRows];  // H[i * kEngRows + j]
};

struct EngItem {
  int slot, idx;
};

// ---- launchers (engine_kernels.cu, engine_ops_*.cu)
struct EngLaunch {
  const EngItem* op_items;
  const int* n_op_items;
  const EngItem* chunk_items;
  const int* n_chunk_items;
  const int* active;  // active slot ids
  int n_active;
  int ctl_threads;  // block size of the controller: 32 kCtlWideWarps when a slot needs the wide reduction
  int op_grid64, op_grid32, chunk_grid;  // residual / Jv grids: the SMs x each kernel's resident blocks
  int* occ;  // prepare only (host): resident blocks per SM of the residual and Jv kernels, [2]
  size_t op_smem64, op_smem32;
  OpArgs<double>* a64;
  OpArgs<float>* a32;
  SlotBuf* buf;
  SlotCtl* ctl;
  double* partials;  // kEngRows per chunk item
  int* tick;         // tick counter (device), advanced by the last launch of a tick
  int any_kron;      // some slot uses the element tensor-product preconditioner
  int any_wide;      // some slot has at least kDotWideLen values
  // global fast-diagonalisation preconditioner: work items (slot, ey s + m) of the x passes and
  // (slot, kx n + jx) of the y/temporal pass, and the shared memory of each pass
  const EngItem* fdm_rows;
  const int* n_fdm_rows;
  const EngItem* fdm_cols;
  const int* n_fdm_cols;
  int any_fdm, fdm_grid_rows, fdm_grid_cols;
  size_t fdm_smem_a, fdm_smem_b, fdm_smem_c;
};

// Launches of the global preconditioner for the slots in kUpdInit / kUpdGSZ (engine_fdm.cu).
cudaError_t eng_fdm_apply(const EngLaunch& L, cudaStream_t st);
// Shared-memory attributes of its kernels (outside stream capture).
cudaError_t eng_fdm_prepare(const EngLaunch& L);

// Whether slot b takes part in the current tick (size-aware sharing: a slot much larger
// than the sharing quantum advances only every stride-th tick).
__device__ __forceinline__ bool eng_runs(const EngLaunch& L, const SlotBuf& b) {
  return b.stride <= 1 || ((*L.tick + b.offset) % b.stride) == 0;
}


// U = 1 (x) uprev, U32 = (float) U for one slot
cudaError_t eng_init_slot(const SlotBuf& b, cudaStream_t st);
// U[i] = U32[i] = state.v[i % r] (a uniform state for tile probing)
struct Fill5 {
  double v[5];
};
cudaError_t eng_fill_state(double* U, float* U32, size_t L, int r, const Fill5& state, cudaStream_t st);
// the launches of one tick after the physics kernels (dot, control, update, tick counter)
cudaError_t eng_tick_tail(const EngLaunch& L, cudaStream_t st);

}  // namespace stdg
