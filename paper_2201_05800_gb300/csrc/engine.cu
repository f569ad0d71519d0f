// Host side of the batched engine (engine.cuh): device arena, slot table,
// work-item lists and the stdg_batch_* entry points of include/stdg.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "args_host.cuh"
#include "lgl_host.h"
#include "engine.cuh"
#include "fdm_host.h"
#include "engine_ops.cuh"
#include "ops.h"
#include "stdg.h"

using namespace stdg;

namespace {

constexpr size_t kAlign = 256;
// values per work item of the build / dot / update kernels: a power of two in [kChunkMin, kChunkMax]
// near L / (4 SMs), so that a slot alone fills the four resident blocks per SM of those kernels in
// about one wave, and a large one keeps few partial sums (it depends on the slot and the device
// only, not on the other slots)
constexpr size_t kChunkMin = 2048, kChunkMax = 65536;
constexpr size_t kOpSmemCap = 96 * 1024;
constexpr size_t kFdmMaxLine = 4096;  // complex values of one x-line group or one y column of the fdm passes

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Best-fit allocator over one device region (offsets, kAlign-aligned sizes).
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes
  void init(size_t bytes) {
    size = bytes;
    free_.clear();
    free_[0] = bytes;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    auto best = free_.end();
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes && (best == free_.end() || it->second < best->second)) best = it;
    if (best == free_.end()) return false;
    *off = best->first;
    const size_t rest = best->second - bytes;
    const size_t roff = best->first + bytes;
    free_.erase(best);
    if (rest) free_[roff] = rest;
    return true;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_bytes() const {
    size_t t = 0;
    for (auto& f : free_) t += f.second;
    return t;
  }
};

struct Layout {
  int n, s, nd, r, m, dim;
  long long nelem;
  size_t L, S, npinv;
  size_t off_U, off_R, off_uprev, off_U32, off_Pinv, off_V, off_Z, off_K, kfloats, bytes;
  // global fast-diagonalisation preconditioner (fdm): eligibility, FFT sizes, data and scratch
  int fdm, kx, ky, ny, logx, logy;
  int f_twx, f_Fx, f_Bx, f_lx, f_twy, f_Fy, f_By, f_ly;
  size_t off_F, ffloats, off_X;
};

struct HostSlot {
  bool used = false, active = false, done = false;
  stdg_config_desc d;
  Layout lay;
  size_t off = 0;
  int epb64 = 1, epb32 = 1;
  SlotBuf buf;
};

}  // namespace

struct stdg_batch {
  stdg_batch_desc d;
  cudaStream_t st = nullptr;
  int device = 0, sms = 1;
  char* arena_base = nullptr;
  Arena arena;
  std::vector<HostSlot> slots;
  // device tables
  SlotCtl* ctl = nullptr;
  OpArgs<double>* a64 = nullptr;
  OpArgs<float>* a32 = nullptr;
  SlotBuf* buf = nullptr;
  int* counts = nullptr;  // [0] op items, [1] chunk items, [2] fdm row items, [3] fdm column items
  EngItem* fdm_rows = nullptr;
  EngItem* fdm_cols = nullptr;
  size_t cap_frows = 0, cap_fcols = 0;
  int n_frows = 0, n_fcols = 0;
  bool any_fdm = false;
  size_t fdm_smem[3] = {0, 0, 0};
  int* active_d = nullptr;
  int* phase_d = nullptr;
  EngItem* op_items = nullptr;
  EngItem* chunk_items = nullptr;
  double* partials = nullptr;
  size_t cap_op = 0, cap_chunk = 0;
  int* phase_h = nullptr;  // pinned
  // host lists
  std::vector<int> active;
  int n_op = 0, n_chunk = 0;
  int max_nitems = 0;  // most chunk items of one active slot (width of the controller blocks)
  bool any_wide = false;  // some active slot takes the 16-row dot pass
  int op_occ[2] = {1, 1};  // resident blocks per SM of the residual and Jv op kernels (set by rebuild)
  bool dirty = true;
  size_t smem64 = 0, smem32 = 0;
  std::string err;
  int* tick_d = nullptr;        // device tick counter
  double share_quantum = 0.0;   // size-aware sharing (0: every slot in every tick)
  int share_max_stride = 16;
  bool use_graphs = true;       // capture the ticks of a step as one CUDA graph
  cudaGraphExec_t gexec = nullptr;
  int gticks = 0;
  bool autotune = false;        // pick elements per CTA of the op kernels by measurement
  bool own_stream = false;      // created here when the caller passed the legacy default stream
  bool any_kron = false;        // some active slot uses the element tensor-product preconditioner
};

namespace {

stdg_status bfail(stdg_batch* b, stdg_status st, const std::string& msg) {
  if (b) b->err = msg;
  return st;
}

#define BCK(b, expr)                                                                                  \
  do {                                                                                                \
    cudaError_t _e = (expr);                                                                          \
    if (_e != cudaSuccess)                                                                            \
      return bfail((b), STDG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));           \
  } while (0)

struct BDev {
  int prev = -1, dev;
  explicit BDev(int d) : dev(d) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~BDev() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
};

int ncomp(int eq, int dim) { return eq == STDG_EULER ? dim + 2 : 1; }

// Measured elements-per-CTA of the two op kernels per problem class (dim, equation, n, s),
// shared by all batches of the process so that a class always gets the same tiles.
struct TuneKey {
  int dim, eq, n, s;
  bool operator<(const TuneKey& o) const {
    return dim != o.dim ? dim < o.dim : eq != o.eq ? eq < o.eq : n != o.n ? n < o.n : s < o.s;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;

bool physics_supported(int dim, int eq) {
  return (eq == STDG_ADVECTION && (dim == 1 || dim == 2)) || (eq == STDG_BURGERS && dim == 2) ||
         (eq == STDG_EULER && dim == 2);
}

stdg_status check_inst(const stdg_batch* b, const stdg_config_desc* d, std::string* why) {
  auto bad = [&](const char* m) { *why = m; return STDG_ERR_INVALID_ARG; };
  if (d->dim != b->d.dim || d->equation != b->d.equation) return bad("dim/equation differ from the batch");
  for (int a = 0; a < d->dim; ++a) {
    if (d->cells[a] < 1) return bad("cells must be >= 1");
    if (!(d->hi[a] > d->lo[a])) return bad("hi must exceed lo");
  }
  if (d->N < 1 || d->N > 7) return bad("N must be 1..7");
  if (d->s < 2 || d->s > 5) return bad("s must be 2..5");
  if (!(d->dt > 0) || !std::isfinite(d->dt)) return bad("dt must be positive");
  if (d->equation == STDG_EULER && !(d->gamma > 1.0)) return bad("gamma must exceed 1");
  if (d->gmres_m < 1 || d->gmres_m > kEngMaxM) return bad("gmres_m must be 1..31");
  if (d->newton_maxit < 1) return bad("newton_maxit must be >= 1");
  if (!(d->newton_rtol >= 0) || !(d->newton_atol >= 0) || !(d->gmres_rtol > 0)) return bad("bad tolerance");
  if (!(d->viscosity >= 0.0) || !std::isfinite(d->viscosity) || !std::isfinite(d->penalty))
    return bad("viscosity must be finite and >= 0");
  if (d->viscosity > 0.0 && d->equation == STDG_EULER) return bad("viscosity is supported for scalar equations");
  return STDG_OK;
}

Layout layout_of(const stdg_config_desc* d) {
  Layout l;
  l.dim = d->dim;
  l.n = d->N + 1;
  l.s = d->s;
  l.r = ncomp(d->equation, d->dim);
  l.m = d->gmres_m;
  l.nd = 1;
  l.nelem = 1;
  for (int a = 0; a < d->dim; ++a) {
    l.nd *= l.n;
    l.nelem *= d->cells[a];
  }
  l.S = (size_t)l.nelem * l.nd * l.r;
  l.L = l.S * l.s;
  // the s x s blocks per spatial node exist only for the point-block preconditioner
  l.npinv = d->precond == STDG_PRECOND_POINT_BLOCK ? (size_t)l.nelem * l.nd * l.s * l.s : 0;
  size_t o = 0;
  l.off_U = o;
  o += align_up(l.L * 8);
  l.off_R = o;
  o += align_up(l.L * 8);
  l.off_uprev = o;
  o += align_up(l.S * 8);
  l.off_U32 = o;
  o += align_up(l.L * 4);
  l.off_Pinv = o;
  o += align_up(l.npinv * 4);
  l.off_V = o;
  o += align_up(l.L * 4 * (size_t)(l.m + 1));
  l.off_Z = o;
  o += align_up(l.L * 4 * (size_t)l.m);
  l.off_K = o;
  l.kfloats = (size_t)4 * l.n * l.n + (size_t)l.nd * l.s * l.s;
  o += align_up(l.kfloats * 4);
  // global preconditioner of scalar slots (not with the point-block option): element counts that
  // are powers of two (radix-2 FFT) and lines that fit the shared-memory tiles of its kernels
  l.fdm = 0;
  l.ffloats = 0;
  l.off_F = l.off_X = o;
  const int kx = d->cells[0], ky = d->dim > 1 ? d->cells[1] : 1;
  auto pow2 = [](int k) { return k >= 1 && (k & (k - 1)) == 0; };
  l.ny = d->dim > 1 ? l.n : 1;
  if (d->equation != STDG_EULER && d->precond != STDG_PRECOND_POINT_BLOCK && d->dim <= 2 && pow2(kx) && pow2(ky) &&
      (size_t)kx * l.n * l.ny <= kFdmMaxLine && (size_t)l.s * ky * l.ny <= kFdmMaxLine) {
    l.fdm = 1;
    l.kx = kx;
    l.ky = ky;
    l.logx = 0;
    while ((1 << l.logx) < kx) ++l.logx;
    l.logy = 0;
    while ((1 << l.logy) < ky) ++l.logy;
    auto even = [](size_t v) { return (int)((v + 1) & ~(size_t)1); };  // complex data on 8-byte boundaries
    int f = 0;
    l.f_twx = f; f += even(2 * kx);
    l.f_Fx = f;  f += even(2 * (size_t)kx * l.n * l.n);
    l.f_Bx = f;  f += even(2 * (size_t)kx * l.n * l.n);
    l.f_lx = f;  f += even((size_t)kx * l.n);
    l.f_twy = f; f += even(2 * ky);
    l.f_Fy = f;  f += even(2 * (size_t)ky * l.ny * l.ny);
    l.f_By = f;  f += even(2 * (size_t)ky * l.ny * l.ny);
    l.f_ly = f;  f += even((size_t)ky * l.ny);
    l.ffloats = f;
    l.off_F = o;
    o += align_up(l.ffloats * 4);
    l.off_X = o;
    o += align_up(l.L * 8);  // one complex value per slab value
  }
  l.bytes = o;
  return l;
}

// Largest elements-per-CTA (<= 256 / n^d nodes per CTA) whose tile fits the cap.
int pick_epb(int dim, int eq, int tsize, int mode, int n, int s, long long nelem, int nd) {
  const int r = ncomp(eq, dim);
  int epb = std::max(1, 256 / nd);
  if (epb > nelem) epb = (int)nelem;
  while (epb > 1 && operator_smem_bytes(dim, r, tsize, mode, n, s, epb) > kOpSmemCap) --epb;
  return epb;
}

template <class T>
cudaError_t grow(T** p, size_t* cap, size_t need, cudaStream_t st) {
  if (need <= *cap) return cudaSuccess;
  size_t nc = std::max(need, *cap * 2 + 64);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  e = cudaMalloc(p, nc * sizeof(T));
  if (e != cudaSuccess) return e;
  *cap = nc;
  return cudaSuccess;
}

cudaError_t physics(stdg_batch* b, const EngLaunch& L, int prepare) {
  if (b->d.equation == STDG_EULER && b->d.dim == 2) return eng_physics_euler2(L, b->st, prepare);
  if (b->d.equation == STDG_BURGERS && b->d.dim == 2) return eng_physics_burgers2(L, b->st, prepare);
  return eng_physics_advection(b->d.dim, L, b->st, prepare);
}

cudaError_t probe(const stdg_batch* b, int mode, const OpArgs<double>& a64, const OpArgs<float>& a32) {
  if (b->d.equation == STDG_EULER && b->d.dim == 2) return eng_probe_euler2(mode, a64, a32, b->st);
  if (b->d.equation == STDG_BURGERS && b->d.dim == 2) return eng_probe_burgers2(mode, a64, a32, b->st);
  return eng_probe_advection(b->d.dim, mode, a64, a32, b->st);
}

// Work-item lists and slot records of the active slots.
stdg_status rebuild(stdg_batch* b) {
  std::vector<EngItem> op, ch, frows, fcols;
  b->smem64 = b->smem32 = 0;
  b->max_nitems = 0;
  b->any_fdm = false;
  b->fdm_smem[0] = b->fdm_smem[1] = b->fdm_smem[2] = 0;
  b->any_kron = false;
  for (int id : b->active) b->any_kron = b->any_kron || b->slots[id].buf.kron;
  b->any_wide = false;
  for (int id : b->active) b->any_wide = b->any_wide || b->slots[id].lay.L >= kDotWideLen;
  for (int id : b->active) {
    HostSlot& hs = b->slots[id];
    const Layout& l = hs.lay;
    const long long tiles = (l.nelem + hs.epb64 - 1) / hs.epb64;
    const long long tiles32 = (l.nelem + hs.epb32 - 1) / hs.epb32;
    // one item list serves both op kernels: tile indices valid for both epb values
    hs.buf.op0 = (int)op.size();
    hs.buf.nop = (int)std::max(tiles, tiles32);
    for (long long t = 0; t < std::max(tiles, tiles32); ++t) op.push_back({id, (int)t});
    hs.buf.item0 = (int)ch.size();
    for (int c = 0; c < hs.buf.nitems; ++c) ch.push_back({id, c});
    b->max_nitems = std::max(b->max_nitems, hs.buf.nitems);
    if (hs.buf.fdm) {
      b->any_fdm = true;
      for (int r = 0; r < l.ky * l.s; ++r) frows.push_back({id, r});
      for (int r = 0; r < l.kx * l.n; ++r) fcols.push_back({id, r});
      const size_t line = (size_t)l.kx * l.n * l.ny, col = (size_t)l.s * l.ky * l.ny;
      b->fdm_smem[0] = std::max(b->fdm_smem[0], line * sizeof(float2));
      b->fdm_smem[1] = std::max(b->fdm_smem[1], 2 * col * sizeof(float2));
      b->fdm_smem[2] = std::max(b->fdm_smem[2], 2 * line * sizeof(float2));
    }
    b->smem64 = std::max(b->smem64, operator_smem_bytes(l.dim, l.r, 8, kModeResidual, l.n, l.s, hs.epb64));
    b->smem32 = std::max(b->smem32, operator_smem_bytes(l.dim, l.r, 4, kModeJvExact, l.n, l.s, hs.epb32));
    BCK(b, cudaMemcpyAsync(b->buf + id, &hs.buf, sizeof(SlotBuf), cudaMemcpyHostToDevice, b->st));
  }
  // size-aware sharing: stride = clamp(round(L / quantum), 1, max_stride); offsets spread the
  // large slots over the ticks of a period
  int next_off = 0;
  for (int id : b->active) {
    HostSlot& hs = b->slots[id];
    int stride = 1;
    if (b->share_quantum > 0.0)
      stride = (int)std::min<double>(b->share_max_stride, std::max(1.0, std::floor(hs.lay.L / b->share_quantum + 0.5)));
    hs.buf.stride = stride;
    hs.buf.offset = stride > 1 ? (next_off++ % stride) : 0;
    BCK(b, cudaMemcpyAsync(b->buf + id, &hs.buf, sizeof(SlotBuf), cudaMemcpyHostToDevice, b->st));
  }
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  BCK(b, grow(&b->op_items, &b->cap_op, std::max<size_t>(op.size(), 1), b->st));
  size_t capc = b->cap_chunk;
  BCK(b, grow(&b->chunk_items, &b->cap_chunk, std::max<size_t>(ch.size(), 1), b->st));
  if (b->cap_chunk != capc || !b->partials) {
    BCK(b, cudaStreamSynchronize(b->st));
    if (b->partials) cudaFree(b->partials);
    b->partials = nullptr;
    BCK(b, cudaMalloc(&b->partials, b->cap_chunk * kEngRows * sizeof(double)));
  }
  if (!op.empty())
    BCK(b, cudaMemcpyAsync(b->op_items, op.data(), op.size() * sizeof(EngItem), cudaMemcpyHostToDevice, b->st));
  if (!ch.empty())
    BCK(b, cudaMemcpyAsync(b->chunk_items, ch.data(), ch.size() * sizeof(EngItem), cudaMemcpyHostToDevice, b->st));
  BCK(b, grow(&b->fdm_rows, &b->cap_frows, std::max<size_t>(frows.size(), 1), b->st));
  BCK(b, grow(&b->fdm_cols, &b->cap_fcols, std::max<size_t>(fcols.size(), 1), b->st));
  if (!frows.empty())
    BCK(b, cudaMemcpyAsync(b->fdm_rows, frows.data(), frows.size() * sizeof(EngItem), cudaMemcpyHostToDevice, b->st));
  if (!fcols.empty())
    BCK(b, cudaMemcpyAsync(b->fdm_cols, fcols.data(), fcols.size() * sizeof(EngItem), cudaMemcpyHostToDevice, b->st));
  int cnt[4] = {(int)op.size(), (int)ch.size(), (int)frows.size(), (int)fcols.size()};
  BCK(b, cudaMemcpyAsync(b->counts, cnt, sizeof(cnt), cudaMemcpyHostToDevice, b->st));
  if (!b->active.empty())
    BCK(b, cudaMemcpyAsync(b->active_d, b->active.data(), b->active.size() * sizeof(int), cudaMemcpyHostToDevice,
                           b->st));
  {
    EngLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.op_smem64 = b->smem64;
    L.op_smem32 = b->smem32;
    L.occ = b->op_occ;
    BCK(b, physics(b, L, 1));
    if (b->any_fdm) {
      L.fdm_smem_a = b->fdm_smem[0];
      L.fdm_smem_b = b->fdm_smem[1];
      L.fdm_smem_c = b->fdm_smem[2];
      BCK(b, eng_fdm_prepare(L));
    }
  }
  // the host vectors are pageable: make the copies complete before they go out of scope
  BCK(b, cudaStreamSynchronize(b->st));
  b->n_op = cnt[0];
  b->n_chunk = cnt[1];
  b->n_frows = cnt[2];
  b->n_fcols = cnt[3];
  b->dirty = false;
  return STDG_OK;
}

// Launches of one tick (the lists must be current).
stdg_status tick(stdg_batch* b) {
  if (b->active.empty()) return STDG_OK;
  EngLaunch L;
  L.op_items = b->op_items;
  L.n_op_items = b->counts;
  L.chunk_items = b->chunk_items;
  L.n_chunk_items = b->counts + 1;
  L.active = b->active_d;
  L.n_active = (int)b->active.size();
  L.ctl_threads = b->max_nitems > kCtlWideItems ? 32 * kCtlWideWarps : kEngThreads;
  L.op_grid64 = std::max(1, std::min(b->n_op, b->sms * std::max(1, b->op_occ[0])));
  L.op_grid32 = std::max(1, std::min(b->n_op, b->sms * std::max(1, b->op_occ[1])));
  L.occ = nullptr;
  L.chunk_grid = std::max(1, std::min(b->n_chunk, b->sms * 8));
  L.op_smem64 = b->smem64;
  L.op_smem32 = b->smem32;
  L.a64 = b->a64;
  L.a32 = b->a32;
  L.buf = b->buf;
  L.ctl = b->ctl;
  L.partials = b->partials;
  L.tick = b->tick_d;
  L.any_kron = b->any_kron ? 1 : 0;
  L.any_wide = b->any_wide ? 1 : 0;
  L.fdm_rows = b->fdm_rows;
  L.n_fdm_rows = b->counts + 2;
  L.fdm_cols = b->fdm_cols;
  L.n_fdm_cols = b->counts + 3;
  L.any_fdm = b->any_fdm ? 1 : 0;
  L.fdm_grid_rows = std::max(1, std::min(b->n_frows, b->sms * 4));
  L.fdm_grid_cols = std::max(1, std::min(b->n_fcols, b->sms * 4));
  L.fdm_smem_a = b->fdm_smem[0];
  L.fdm_smem_b = b->fdm_smem[1];
  L.fdm_smem_c = b->fdm_smem[2];
  cudaError_t e = physics(b, L, 0);
  if (e != cudaSuccess) return bfail(b, STDG_ERR_CUDA, std::string("engine physics launch: ") + cudaGetErrorString(e));
  e = eng_tick_tail(L, b->st);
  if (e != cudaSuccess) return bfail(b, STDG_ERR_CUDA, std::string("engine launch: ") + cudaGetErrorString(e));
  return STDG_OK;
}

__global__ void gather_phase_kernel(const int* active, int n, const SlotCtl* ctl, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ctl[active[i]].phase;
}

// Drop finished slots from the active list; *working = slots still working.
stdg_status refresh(stdg_batch* b, int* working) {
  const int n = (int)b->active.size();
  if (n > 0) {
    gather_phase_kernel<<<(n + 255) / 256, 256, 0, b->st>>>(b->active_d, n, b->ctl, b->phase_d);
    BCK(b, cudaGetLastError());
    BCK(b, cudaMemcpyAsync(b->phase_h, b->phase_d, n * sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BCK(b, cudaStreamSynchronize(b->st));
    std::vector<int> keep;
    for (int i = 0; i < n; ++i) {
      const int id = b->active[i];
      if (b->phase_h[i] == kPhDone) {
        b->slots[id].active = false;
        b->slots[id].done = true;
        b->dirty = true;
      } else {
        keep.push_back(id);
      }
    }
    b->active.swap(keep);
  }
  if (working) *working = (int)b->active.size();
  return STDG_OK;
}

// Eigen-decomposition of a symmetric n x n matrix S (row major, destroyed) by cyclic Jacobi
// rotations (Golub and Van Loan, Sec. 8.5): S = Q diag(lam) Q^T, Q row major.
void sym_eig(int n, double* S, double* Q, double* lam) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Q[i * n + j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += S[i * n + j] * S[i * n + j];
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = S[p * n + q];
        if (apq == 0.0) continue;
        const double theta = (S[q * n + q] - S[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // S <- S J
          const double skp = S[k * n + p], skq = S[k * n + q];
          S[k * n + p] = c * skp - sn * skq;
          S[k * n + q] = sn * skp + c * skq;
        }
        for (int k = 0; k < n; ++k) {  // S <- J^T S
          const double spk = S[p * n + k], sqk = S[q * n + k];
          S[p * n + k] = c * spk - sn * sqk;
          S[q * n + k] = sn * spk + c * sqk;
        }
        for (int k = 0; k < n; ++k) {  // Q <- Q J
          const double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - sn * qkq;
          Q[k * n + q] = sn * qkp + c * qkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = S[i * n + i];
}

// Inverse of an s x s matrix (row major) by Gauss-Jordan with partial pivoting.
void small_inverse(int s, const double* A, double* Ai) {
  double W[kMaxS][2 * kMaxS];
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      W[i][j] = A[i * s + j];
      W[i][s + j] = i == j ? 1.0 : 0.0;
    }
  for (int c = 0; c < s; ++c) {
    int pv = c;
    for (int q = c + 1; q < s; ++q)
      if (std::fabs(W[q][c]) > std::fabs(W[pv][c])) pv = q;
    for (int j = 0; j < 2 * s; ++j) std::swap(W[c][j], W[pv][j]);
    const double inv = 1.0 / W[c][c];
    for (int j = 0; j < 2 * s; ++j) W[c][j] *= inv;
    for (int q = 0; q < s; ++q)
      if (q != c) {
        const double f = W[q][c];
        for (int j = 0; j < 2 * s; ++j) W[q][j] -= f * W[c][j];
      }
  }
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) Ai[i * s + j] = W[i][s + j];
}

// Data of the element tensor-product preconditioner of a scalar slot (see eng_kron_kernel):
// the element-local 1D operators A_a (interior penalty form with the neighbours zero, plus
// the upwind dissipation lambda_a/(h_a w_end) at both end nodes, lambda_a the slot's wave
// speed bound), their eigen-decompositions (A_a = W^-1 K_a with K_a symmetric, so
// A_a = V Lambda V^-1, V = W^-1/2 Q, V^-1 = Q^T W^1/2) and P_k^-1 = (T - dt/2 Lambda_k M_tau)^-1
// for every mode k of the element.
std::vector<float> kron_data(const stdg_config_desc* d, int n, int s, int nd, const double lam[3]) {
  const int N = n - 1, dim = d->dim;
  double xi[16], w[16], D[256], tau[16], om[16], Dt[256];
  lgl_rule(n, xi, w);
  diff_matrix(n, xi, D);
  lgl_rule(s, tau, om);
  diff_matrix(s, tau, Dt);
  const double nu = d->viscosity;
  const double eta = d->penalty > 0.0 ? d->penalty : 10.0 * N * N;
  std::vector<double> V[2], Vi[2], lm[2];
  for (int a = 0; a < 2; ++a) {
    V[a].assign(n * n, 0.0);
    Vi[a].assign(n * n, 0.0);
    lm[a].assign(n, 0.0);
    for (int i = 0; i < n; ++i) V[a][i * n + i] = Vi[a][i * n + i] = 1.0;
    if (a >= dim) continue;
    const double h = (d->hi[a] - d->lo[a]) / d->cells[a], g = 2.0 / h, sig = nu * eta / h;
    std::vector<double> A(n * n, 0.0);
    for (int i = 0; i < n; ++i) {  // column i: response to the unit vector e_i
      std::vector<double> q(n), B(n, 0.0);
      for (int k = 0; k < n; ++k) q[k] = g * D[k * n + i];
      for (int ip = 0; ip < n; ++ip) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += w[k] * D[k * n + ip] * q[k];
        B[ip] = nu * g / w[ip] * acc;
      }
      const double jup = i == N ? 1.0 : 0.0, jlo = i == 0 ? -1.0 : 0.0;
      B[N] += g / w[N] * (-nu * 0.5 * q[N] + sig * jup);
      B[0] += g / w[0] * (nu * 0.5 * q[0] - sig * jlo);
      for (int ip = 0; ip < n; ++ip) B[ip] -= g / w[ip] * nu * 0.5 * g * (D[N * n + ip] * jup + D[ip] * jlo);
      if (i == N) B[N] += 0.5 * g / w[N] * lam[a];
      if (i == 0) B[0] += 0.5 * g / w[0] * lam[a];
      for (int ip = 0; ip < n; ++ip) A[ip * n + i] = B[ip];
    }
    std::vector<double> S(n * n), Q(n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double sij = std::sqrt(w[i]) * A[i * n + j] / std::sqrt(w[j]);
        const double sji = std::sqrt(w[j]) * A[j * n + i] / std::sqrt(w[i]);
        S[i * n + j] = 0.5 * (sij + sji);
      }
    sym_eig(n, S.data(), Q.data(), lm[a].data());
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < n; ++k) {
        V[a][i * n + k] = Q[i * n + k] / std::sqrt(w[i]);
        Vi[a][k * n + i] = Q[i * n + k] * std::sqrt(w[i]);
      }
  }
  std::vector<float> out((size_t)4 * n * n + (size_t)nd * s * s);
  for (int i = 0; i < n * n; ++i) {
    out[i] = (float)Vi[0][i];
    out[n * n + i] = (float)V[0][i];
    out[2 * n * n + i] = (float)Vi[1][i];
    out[3 * n * n + i] = (float)V[1][i];
  }
  std::vector<double> P(s * s), Pi(s * s);
  for (int k = 0; k < nd; ++k) {
    const double Lk = lm[0][k % n] + (dim > 1 ? lm[1][(k / n) % n] : 0.0);
    for (int m = 0; m < s; ++m)
      for (int j = 0; j < s; ++j) {
        double v = om[j] * Dt[j * s + m];  // (D_tau^T M_tau)[m][j]
        if (m == s - 1 && j == s - 1) v -= 1.0;
        if (m == j) v -= 0.5 * d->dt * Lk * om[m];
        P[m * s + j] = v;
      }
    small_inverse(s, P.data(), Pi.data());
    for (int q = 0; q < s * s; ++q) out[(size_t)4 * n * n + (size_t)k * s * s + q] = (float)Pi[q];
  }
  return out;
}

// Data of the global fast-diagonalisation preconditioner of a scalar slot (see engine_fdm.cu):
// twiddles exp(-2 pi i t / K), the per-mode transforms F_k, B_k and eigenvalues of the periodic
// 1D operator along x and y (fdm_host.h), as FP32 at the offsets of the layout.
bool fdm_data(const stdg_config_desc* d, const Layout& l, const double lam[3], std::vector<float>* out) {
  out->assign(l.ffloats, 0.0f);
  float* o = out->data();
  const double pi = 3.14159265358979323846;
  double xi[16], w[16];
  lgl_rule(l.n, xi, w);
  const int dims[2] = {l.kx, l.ky};
  const int offs[2][4] = {{l.f_twx, l.f_Fx, l.f_Bx, l.f_lx}, {l.f_twy, l.f_Fy, l.f_By, l.f_ly}};
  for (int a = 0; a < 2; ++a) {
    const int K = dims[a];
    for (int t = 0; t < K; ++t) {
      o[offs[a][0] + 2 * t] = (float)std::cos(2.0 * pi * t / K);
      o[offs[a][0] + 2 * t + 1] = (float)-std::sin(2.0 * pi * t / K);
    }
    if (a == 1 && d->dim == 1) {  // no y direction: identity transforms, eigenvalue 0
      o[offs[a][1]] = o[offs[a][2]] = 1.0f;
      o[offs[a][3]] = 0.0f;
      continue;
    }
    const int n = l.n;
    const double h = (d->hi[a] - d->lo[a]) / d->cells[a];
    std::vector<double> A0(n * n), Ap(n * n), Am(n * n), lmb((size_t)K * n);
    std::vector<cplx> B((size_t)K * n * n), F((size_t)K * n * n);
    fdm_blocks_1d(n, h, d->viscosity, d->penalty, lam[a], A0.data(), Ap.data(), Am.data());
    if (!fdm_symbol_eig(n, K, A0.data(), Ap.data(), Am.data(), w, lmb.data(), B.data(), F.data())) return false;
    for (size_t i = 0; i < B.size(); ++i) {
      o[offs[a][1] + 2 * i] = (float)F[i].real();
      o[offs[a][1] + 2 * i + 1] = (float)F[i].imag();
      o[offs[a][2] + 2 * i] = (float)B[i].real();
      o[offs[a][2] + 2 * i + 1] = (float)B[i].imag();
    }
    for (size_t i = 0; i < lmb.size(); ++i) o[offs[a][3] + i] = (float)lmb[i];
  }
  return true;
}

// Elements per CTA of the two op kernels for the slot's class: cached, else measured.  The
// probe is a virtual periodic grid of the class with at least 4096 elements (enough CTAs to
// fill the GPU, as in a loaded batch) holding a uniform state; each candidate tile is timed
// over three launches after a warm-up, and the fastest kept (the smaller tile unless the
// larger is more than 3% faster).
stdg_status tune(stdg_batch* b, const Layout& l, int eq, const OpArgs<double>& k64, const OpArgs<float>& k32,
                 int* epb64, int* epb32) {
  const TuneKey key{l.dim, eq, l.n, l.s};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *epb64 = it->second.first;
      *epb32 = it->second.second;
      return STDG_OK;
    }
  }
  const int r = ncomp(eq, l.dim);
  const int side = l.dim == 1 ? 4096 : 64;
  const long long nel = l.dim == 1 ? 4096 : 4096;
  const size_t S = (size_t)nel * l.nd * r, L = S * l.s;
  double *U = nullptr, *R = nullptr, *up = nullptr;
  float *U32 = nullptr, *O32 = nullptr;
  bool ok = cudaMalloc(&U, L * 8) == cudaSuccess && cudaMalloc(&R, L * 8) == cudaSuccess &&
            cudaMalloc(&up, S * 8) == cudaSuccess && cudaMalloc(&U32, L * 4) == cudaSuccess &&
            cudaMalloc(&O32, L * 4) == cudaSuccess;
  Fill5 st;
  if (eq == STDG_EULER) {
    const double rho = 1.0, v = 0.5, p = 1.0;
    st.v[0] = rho;
    for (int a = 0; a < l.dim; ++a) st.v[1 + a] = rho * v;
    st.v[r - 1] = p / (k64.gamma - 1.0) + 0.5 * rho * v * v * l.dim;
  } else {
    st.v[0] = 0.3;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ok = ok && eng_fill_state(U, U32, L, r, st, b->st) == cudaSuccess &&
       cudaMemcpyAsync(up, U, S * 8, cudaMemcpyDeviceToDevice, b->st) == cudaSuccess &&
       cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  int best[2] = {*epb64, *epb32};
  if (ok) {
    const int maxe = std::max(1, 256 / l.nd);
    const int cand[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 28, 32};
    for (int mode = 0; mode < 2 && ok; ++mode) {
      float best_ms = 1e30f;
      for (int c : cand) {
        if (c > maxe) break;
        if (operator_smem_bytes(l.dim, r, mode == 0 ? 8 : 4, mode == 0 ? kModeResidual : kModeJvExact, l.n, l.s,
                                c) > kOpSmemCap)
          break;
        OpArgs<double> a = k64;
        OpArgs<float> f = k32;
        a.K[0] = f.K[0] = l.dim == 1 ? (int)nel : side;
        a.K[1] = f.K[1] = l.dim == 1 ? 1 : side;
        a.K[2] = f.K[2] = 1;
        a.nelem = f.nelem = nel;
        a.epb = f.epb = c;
        a.U = U;
        a.uprev = up;
        a.out = R;
        a.fout = nullptr;
        f.U = U32;
        f.v = U32;
        f.out = O32;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 4 && ok; ++rep) {
          ok = cudaEventRecord(e0, b->st) == cudaSuccess && probe(b, mode, a, f) == cudaSuccess &&
               cudaEventRecord(e1, b->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
          float ms = 0.f;
          if (ok) cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) ms_min = std::min(ms_min, ms);  // the first launch warms up
        }
        if (ms_min < best_ms * 0.97f) {
          best_ms = ms_min;
          best[mode] = c;
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(U);
  cudaFree(R);
  cudaFree(up);
  cudaFree(U32);
  cudaFree(O32);
  if (!ok) {
    cudaGetLastError();
    return bfail(b, STDG_ERR_CUDA, "tile probing failed");
  }
  // a tile larger than the slot is clipped by the slot (fewer elements than one tile)
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto ins = g_tune.emplace(key, std::make_pair(best[0], best[1]));
  *epb64 = ins.first->second.first;
  *epb32 = ins.first->second.second;
  return STDG_OK;
}

}  // namespace

extern "C" {

stdg_status stdg_batch_create(const stdg_batch_desc* desc, void* cuda_stream, stdg_batch** out) {
  if (!out) return STDG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || desc->max_slots < 1 || desc->hbm_budget_bytes == 0 || !physics_supported(desc->dim, desc->equation))
    return STDG_ERR_INVALID_ARG;
  stdg_batch* b = new stdg_batch();
  b->d = *desc;
  b->st = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return STDG_ERR_CUDA;
  }
  if (!b->st) {
    // graph capture needs a stream of its own; every batch call returns after its work
    // completed, so the caller sees the same ordering as on the default stream
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return STDG_ERR_CUDA;
    }
    b->own_stream = true;
  }
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (b->sms < 1) b->sms = 1;
  const int ns = desc->max_slots;
  b->slots.resize(ns);
  bool ok = cudaMalloc(&b->arena_base, desc->hbm_budget_bytes) == cudaSuccess;
  ok = ok && cudaMalloc(&b->ctl, ns * sizeof(SlotCtl)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->a64, ns * sizeof(OpArgs<double>)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->a32, ns * sizeof(OpArgs<float>)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->buf, ns * sizeof(SlotBuf)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->counts, 4 * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->active_d, ns * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->phase_d, ns * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->phase_h, ns * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->tick_d, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    stdg_batch_destroy(b);
    return STDG_ERR_OOM;
  }
  if (cudaMemsetAsync(b->ctl, 0, ns * sizeof(SlotCtl), b->st) != cudaSuccess ||
      cudaMemsetAsync(b->counts, 0, 4 * sizeof(int), b->st) != cudaSuccess ||
      cudaMemsetAsync(b->tick_d, 0, sizeof(int), b->st) != cudaSuccess ||
      cudaStreamSynchronize(b->st) != cudaSuccess) {
    cudaGetLastError();
    stdg_batch_destroy(b);
    return STDG_ERR_CUDA;
  }
  b->arena.init(desc->hbm_budget_bytes);
  *out = b;
  return STDG_OK;
}

stdg_status stdg_batch_destroy(stdg_batch* b) {
  if (!b) return STDG_ERR_INVALID_ARG;
  BDev g(b->device);
  cudaStreamSynchronize(b->st);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  void* ps[] = {b->arena_base, b->ctl, b->a64, b->a32, b->buf, b->counts, b->active_d, b->phase_d,
                b->op_items, b->chunk_items, b->partials, b->tick_d, b->fdm_rows, b->fdm_cols};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (b->phase_h) cudaFreeHost(b->phase_h);
  if (b->own_stream) cudaStreamDestroy(b->st);
  cudaGetLastError();
  delete b;
  return STDG_OK;
}

size_t stdg_batch_slot_bytes(const stdg_batch* b, const stdg_config_desc* inst) {
  if (!b || !inst) return 0;
  std::string why;
  if (check_inst(b, inst, &why) != STDG_OK) return 0;
  return layout_of(inst).bytes;
}

size_t stdg_batch_free_bytes(const stdg_batch* b) { return b ? b->arena.free_bytes() : 0; }

stdg_status stdg_batch_add(stdg_batch* b, const stdg_config_desc* d, const double* u0, int kind, int* slot) {
  if (!b || !d || !u0 || !slot || (kind != STDG_HOST && kind != STDG_DEVICE)) return STDG_ERR_INVALID_ARG;
  *slot = -1;
  std::string why;
  if (check_inst(b, d, &why) != STDG_OK) return bfail(b, STDG_ERR_INVALID_ARG, why);
  BDev g(b->device);
  int id = -1;
  for (int i = 0; i < (int)b->slots.size(); ++i)
    if (!b->slots[i].used) {
      id = i;
      break;
    }
  if (id < 0) return bfail(b, STDG_ERR_OOM, "slot table full");
  const Layout l = layout_of(d);
  size_t off;
  if (!b->arena.alloc(l.bytes, &off)) return bfail(b, STDG_ERR_OOM, "arena full");
  HostSlot& hs = b->slots[id];
  hs = HostSlot();
  hs.used = true;
  hs.active = true;
  hs.d = *d;
  hs.lay = l;
  hs.off = off;
  char* base = b->arena_base + off;
  SlotBuf& sb = hs.buf;
  sb.U = reinterpret_cast<double*>(base + l.off_U);
  sb.R = reinterpret_cast<double*>(base + l.off_R);
  sb.uprev = reinterpret_cast<double*>(base + l.off_uprev);
  sb.U32 = reinterpret_cast<float*>(base + l.off_U32);
  sb.Pinv = reinterpret_cast<float*>(base + l.off_Pinv);
  sb.V = reinterpret_cast<float*>(base + l.off_V);
  sb.Z = reinterpret_cast<float*>(base + l.off_Z);
  sb.nelem = l.nelem;
  sb.s = l.s;
  sb.nd = l.nd;
  sb.r = l.r;
  sb.L = l.L;
  size_t chunk = kChunkMin;
  while (chunk < kChunkMax && chunk < l.L / (4 * (size_t)b->sms)) chunk <<= 1;
  sb.chunk_elems = std::max(1, (int)(chunk / ((size_t)l.s * l.nd * l.r)));
  sb.nitems = (int)((l.nelem + sb.chunk_elems - 1) / sb.chunk_elems);
  sb.item0 = 0;
  sb.op0 = sb.nop = 0;
  sb.vec4 = l.L % 4 == 0 ? 1 : 0;
  sb.dim = l.dim;
  sb.n = l.n;
  sb.kron = (d->equation != STDG_EULER && d->precond != STDG_PRECOND_POINT_BLOCK) ? 1 : 0;
  sb.pbtm = (d->equation == STDG_EULER && d->precond != STDG_PRECOND_POINT_BLOCK) ? 1 : 0;
  sb.kdat = reinterpret_cast<const float*>(base + l.off_K);
  sb.fdm = 0;
  sb.fkx = l.kx;
  sb.fky = l.ky;
  sb.fny = l.ny;
  sb.flogx = l.logx;
  sb.flogy = l.logy;
  sb.f_twx = l.f_twx;
  sb.f_Fx = l.f_Fx;
  sb.f_Bx = l.f_Bx;
  sb.f_lx = l.f_lx;
  sb.f_twy = l.f_twy;
  sb.f_Fy = l.f_Fy;
  sb.f_By = l.f_By;
  sb.f_ly = l.f_ly;
  sb.fdat = reinterpret_cast<const float*>(base + l.off_F);
  sb.fx = reinterpret_cast<float2*>(base + l.off_X);
  if (sb.kron) {
    double lam[3] = {0.0, 0.0, 0.0};
    if (d->equation == STDG_ADVECTION) {
      for (int a = 0; a < 3; ++a) lam[a] = std::fabs(d->adv_vel[a]);
    } else {  // Burgers: the largest |u| of the initial state bounds the wave speed
      std::vector<double> hu;
      const double* u = u0;
      if (kind == STDG_DEVICE) {
        hu.resize(l.S);
        BCK(b, cudaMemcpy(hu.data(), u0, l.S * sizeof(double), cudaMemcpyDeviceToHost));
        u = hu.data();
      }
      double mx = 0.0;
      for (size_t i = 0; i < l.S; ++i) mx = std::max(mx, std::fabs(u[i]));
      lam[0] = lam[1] = lam[2] = mx;
    }
    std::vector<float> kd = kron_data(d, l.n, l.s, l.nd, lam);
    BCK(b, cudaMemcpy(base + l.off_K, kd.data(), kd.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (l.fdm) {
      std::vector<float> fd;
      if (!fdm_data(d, l, lam, &fd)) return bfail(b, STDG_ERR_NOT_CONVERGED, "fdm: eigensolve did not converge");
      BCK(b, cudaMemcpy(base + l.off_F, fd.data(), fd.size() * sizeof(float), cudaMemcpyHostToDevice));
      sb.kron = 0;
      sb.fdm = 1;
    }
  }
  hs.epb64 = pick_epb(l.dim, d->equation, 8, kModeResidual, l.n, l.s, l.nelem, l.nd);
  hs.epb32 = pick_epb(l.dim, d->equation, 4, kModeJvExact, l.n, l.s, l.nelem, l.nd);
  // operator constants
  double h[3] = {1, 1, 1};
  for (int a = 0; a < l.dim; ++a) h[a] = (d->hi[a] - d->lo[a]) / d->cells[a];
  OpArgs<double> k64;
  OpArgs<float> k32;
  fill_op_args<double>(k64, l.dim, l.n, l.s, d->cells, h, d->dt, d->gamma, d->adv_vel, d->viscosity, d->penalty);
  fill_op_args<float>(k32, l.dim, l.n, l.s, d->cells, h, d->dt, d->gamma, d->adv_vel, d->viscosity, d->penalty);
  k64.epb = hs.epb64;
  k64.U = sb.U;
  k64.uprev = sb.uprev;
  k64.out = sb.R;
  k64.fout = nullptr;
  k32.epb = hs.epb32;
  k32.U = sb.U32;
  k32.v = sb.Z;
  k32.out = sb.V + l.L;
  k32.vscale = 1.0f;
  k32.lscale = 0;
  SlotCtl c;
  std::memset(&c, 0, sizeof(c));
  c.phase = kPhResid;
  c.m = l.m;
  // each cycle of at most m FGMRES iterations ends with a re-linearisation; the cap on cycles gives
  // a slot the GMRES-iteration budget of the single-slab solver, newton_maxit x gmres_maxit
  c.newton_maxit = d->newton_maxit * std::max(1, (d->gmres_maxit + l.m - 1) / l.m);
  c.rtol = d->newton_rtol;
  c.atol = d->newton_atol;
  c.gmres_rtol = d->gmres_rtol;
  c.status = STDG_OK;
  BCK(b, cudaMemcpyAsync(b->a64 + id, &k64, sizeof(k64), cudaMemcpyHostToDevice, b->st));
  BCK(b, cudaMemcpyAsync(b->a32 + id, &k32, sizeof(k32), cudaMemcpyHostToDevice, b->st));
  BCK(b, cudaMemcpyAsync(b->ctl + id, &c, sizeof(c), cudaMemcpyHostToDevice, b->st));
  BCK(b, cudaMemcpyAsync(sb.uprev, u0, l.S * sizeof(double),
                         kind == STDG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, b->st));
  BCK(b, eng_init_slot(sb, b->st));
  if (b->autotune) {
    stdg_status ts = tune(b, l, d->equation, k64, k32, &hs.epb64, &hs.epb32);
    if (ts != STDG_OK) return ts;
    hs.epb64 = (int)std::min<long long>(hs.epb64, l.nelem);
    hs.epb32 = (int)std::min<long long>(hs.epb32, l.nelem);
    k64.epb = hs.epb64;
    k32.epb = hs.epb32;
    BCK(b, cudaMemcpyAsync(b->a64 + id, &k64, sizeof(k64), cudaMemcpyHostToDevice, b->st));
    BCK(b, cudaMemcpyAsync(b->a32 + id, &k32, sizeof(k32), cudaMemcpyHostToDevice, b->st));
  }
  // the staging structs live on this stack frame
  BCK(b, cudaStreamSynchronize(b->st));
  b->active.push_back(id);
  b->dirty = true;
  *slot = id;
  return STDG_OK;
}

stdg_status stdg_batch_step(stdg_batch* b, int ticks, int* working) {
  if (!b || ticks < 1) return STDG_ERR_INVALID_ARG;
  BDev g(b->device);
  if (b->dirty) {
    stdg_status s = rebuild(b);
    if (s != STDG_OK) return s;
  }
  if (!b->active.empty()) {
    if (b->use_graphs) {
      if (!b->gexec || b->gticks != ticks) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        BCK(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        stdg_status s = STDG_OK;
        for (int t = 0; t < ticks && s == STDG_OK; ++t) s = tick(b);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(b->st, &graph);
        if (s != STDG_OK) {
          if (graph) cudaGraphDestroy(graph);
          return s;
        }
        BCK(b, ce);
        const cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        BCK(b, ie);
        b->gticks = ticks;
      }
      BCK(b, cudaGraphLaunch(b->gexec, b->st));
    } else {
      for (int t = 0; t < ticks; ++t) {
        stdg_status s = tick(b);
        if (s != STDG_OK) return s;
      }
    }
  }
  return refresh(b, working);
}

stdg_status stdg_batch_configure(stdg_batch* b, double share_quantum, int share_max_stride, int use_graphs,
                                 int autotune) {
  if (!b || !(share_quantum >= 0.0) || share_max_stride < 1) return STDG_ERR_INVALID_ARG;
  b->share_quantum = share_quantum;
  b->share_max_stride = share_max_stride;
  b->use_graphs = use_graphs != 0;
  b->autotune = autotune != 0;
  b->dirty = true;
  return STDG_OK;
}

stdg_status stdg_batch_run(stdg_batch* b, int max_ticks, int* working) {
  if (!b || max_ticks < 1) return STDG_ERR_INVALID_ARG;
  int done_ticks = 0, w = (int)b->active.size();
  while (w > 0 && done_ticks < max_ticks) {
    const int t = std::min(8, max_ticks - done_ticks);
    stdg_status s = stdg_batch_step(b, t, &w);
    if (s != STDG_OK) return s;
    done_ticks += t;
  }
  if (working) *working = w;
  return STDG_OK;
}

stdg_status stdg_batch_query(stdg_batch* b, int slot, int* done, int* status, stdg_slab_stats* stats) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return STDG_ERR_INVALID_ARG;
  BDev g(b->device);
  SlotCtl c;
  BCK(b, cudaMemcpyAsync(&c, b->ctl + slot, sizeof(c), cudaMemcpyDeviceToHost, b->st));
  BCK(b, cudaStreamSynchronize(b->st));
  if (done) *done = c.phase == kPhDone ? 1 : 0;
  if (status) *status = c.status;
  if (stats) {
    stats->newton_its = c.newton_its;
    stats->gmres_its = c.gmres_its;
    stats->residual_evals = c.resid_evals;
    stats->jv_evals = c.jv_evals;
    stats->res0 = c.res0;
    stats->res_final = c.res;
  }
  return STDG_OK;
}

stdg_status stdg_batch_get_state(stdg_batch* b, int slot, double* u, int kind) {
  if (!b || !u || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used ||
      (kind != STDG_HOST && kind != STDG_DEVICE))
    return STDG_ERR_INVALID_ARG;
  BDev g(b->device);
  const HostSlot& hs = b->slots[slot];
  BCK(b, cudaMemcpyAsync(u, hs.buf.uprev, hs.lay.S * sizeof(double),
                         kind == STDG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->st));
  BCK(b, cudaStreamSynchronize(b->st));
  return STDG_OK;
}

stdg_status stdg_batch_get_slab(stdg_batch* b, int slot, double* U, int kind) {
  if (!b || !U || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used ||
      (kind != STDG_HOST && kind != STDG_DEVICE))
    return STDG_ERR_INVALID_ARG;
  BDev g(b->device);
  const HostSlot& hs = b->slots[slot];
  BCK(b, cudaMemcpyAsync(U, hs.buf.U, hs.lay.L * sizeof(double),
                         kind == STDG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->st));
  BCK(b, cudaStreamSynchronize(b->st));
  return STDG_OK;
}

stdg_status stdg_batch_remove(stdg_batch* b, int slot) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return STDG_ERR_INVALID_ARG;
  BDev g(b->device);
  // kernels of earlier ticks may still read the slot's memory
  BCK(b, cudaStreamSynchronize(b->st));
  HostSlot& hs = b->slots[slot];
  if (hs.active) {
    b->active.erase(std::find(b->active.begin(), b->active.end(), slot));
    b->dirty = true;
  }
  b->arena.release(hs.off, hs.lay.bytes);
  hs = HostSlot();
  return STDG_OK;
}

int stdg_batch_done_slots(const stdg_batch* b, int* slots, int cap) {
  if (!b) return 0;
  int n = 0;
  for (int i = 0; i < (int)b->slots.size(); ++i)
    if (b->slots[i].used && b->slots[i].done) {
      if (slots && n < cap) slots[n] = i;
      ++n;
    }
  return n;
}

const char* stdg_batch_last_error(const stdg_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
