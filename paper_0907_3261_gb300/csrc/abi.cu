// C-ABI of the library (declared in include/bbicggr.h): context creation, Y = A X, the Jacobi
// preconditioner, and the preconditioned block BiCGGR driver of arXiv:0907.3261, Sec. 2.
//
// The driver keeps every L x L quantity on the device (SolverState) and launches the iteration as
// a fixed sequence of kernels on the caller's stream.  The host reads back L residual norms and a
// status word once per outer iteration, right after the R update, where the stopping test of the
// algorithm box sits; a singular L x L system makes the later kernels of the iteration leave X and
// R untouched, so the returned iterate is the last consistent one.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <initializer_list>
#include <new>
#include <vector>

#include "../../include/bbicggr.h"
#include "internal.h"

namespace {

thread_local char g_err[512] = "";

void set_err(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

#define CU(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? WD_ENOMEM : WD_ECUDA;                  \
    }                                                                                 \
  } while (0)

// Launch under the per-kernel instrumentation (needs `c` and `s` in scope).
#define LAUNCH(cls, nkernels, call)         \
  do {                                      \
    Timed timed_(c, cls, nkernels, s);      \
    CU(call);                               \
  } while (0)

#define CHECK(rc)              \
  do {                         \
    int rc_ = (rc);            \
    if (rc_ != WD_OK) return rc_; \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t need) {
    if (bytes >= need) return WD_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    CU(cudaMalloc(&p, need));
    bytes = need;
    return WD_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  double* d() const { return static_cast<double*>(p); }
};

// Host mirror of what the driver reads back each iteration.
struct HostMirror {
  double rnorm2[WD_LMAX];
  int status;
};

}  // namespace

struct Prof {
  bool timing = false;
  long long kernels[WD_K_COUNT] = {};
  double ms[WD_K_COUNT] = {};
  struct Pending {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
};

struct wd_ctx {
  Op op{};
  Prof prof;
  int device = 0;
  // solver workspace for the current L
  int L = 0;
  int solved_L = 0;        // L of the last solve, whose recursive residual is in blk[B_R]
  DevBuf blk[13];          // R P V W F U G Y Rt T (always); B Xs X0 (on demand)
  DevBuf part;             // reduction partials
  SolverState* st = nullptr;
  HostMirror* hm = nullptr;
  double* bnorm2_dev = nullptr;
  // staging for host pointers in wd_apply / jacobi_precond
  DevBuf stage_in, stage_out;
  // low-precision preconditioner blocks: U and two sweep buffers (sized for FP32 elements)
  DevBuf blk32[3];
  // autotuned tile of the low-precision sweep per storage (LP_F32, LP_BF16, LP_DF) and L: RHS per
  // thread, threads per CTA, min CTAs per SM, shared-memory staging
  int tile_r[3][WD_LMAX + 1] = {};
  int tile_block[3][WD_LMAX + 1] = {};
  int tile_minb[3][WD_LMAX + 1] = {};
  int tile_staged[3][WD_LMAX + 1] = {};
  bool tile_set[3][WD_LMAX + 1] = {};
  bool links_su3 = false;         // the links are special unitary to LINK12_TOL
  wd_net* active_net = nullptr;   // learned preconditioner of the running solve (mode 2)
  bool net_bf16 = false;          // ... with its activations stored in BF16 (precision 3)
  // device-controlled (graph) solves
  void* gctl = nullptr;           // GraphCtl
  double* ghist = nullptr;        // residual history, ghist_len entries
  int ghist_len = 0;
  cudaStream_t capture_stream = nullptr;
  // domain decomposition (wd_set_domain): this context is one rank's t-slab with one halo slice on
  // each side; halo exchanges and sums over ranks go through the caller's callbacks
  bool dom_on = false;
  wd_domain dom{};
  void* dom_host = nullptr;        // pinned staging: 4 halo slices, then the reduction buffer
  size_t dom_host_bytes = 0;
};

namespace {

// Preconditioner modes of precondition(): FP64 sweeps, FP32-storage sweeps, the learned network,
// BF16-storage sweeps, double-float sweeps.
enum { PM_F64 = 0, PM_F32 = 1, PM_NET = 2, PM_BF16 = 3, PM_DF = 4 };

inline int lp_storage(int mode) { return mode == PM_BF16 ? LP_BF16 : LP_F32; }
// Mode for the public options: precision 1 and 2 sweep in FP32, 3 in BF16, 4 and 5 in
// double-float; a network wins.
inline int precond_mode(const bbicggr_opts& o) {
  if (o.net) return PM_NET;
  if (o.precision == 3) return PM_BF16;
  if (o.precision == 4 || o.precision == 5) return PM_DF;
  return o.precision >= 1 ? PM_F32 : PM_F64;
}

enum { B_R, B_P, B_V, B_W, B_F, B_U, B_G, B_Y, B_RT, B_T, B_CORE,
       B_B = B_CORE, B_XS, B_X0, B_COUNT };

size_t block_bytes(const wd_ctx* c, int L) { return (size_t)c->op.g.V * 12 * L * 16; }

cudaEvent_t prof_event(wd_ctx* c) {
  if (!c->prof.pool.empty()) {
    cudaEvent_t e = c->prof.pool.back();
    c->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Counts the kernels of one launcher call of class `cls` and, with timing on, brackets them with
// two events on the launching stream.
struct Timed {
  wd_ctx* c;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Timed(wd_ctx* c_, int cls_, int nkernels, cudaStream_t s_) : c(c_), cls(cls_), s(s_) {
    c->prof.kernels[cls] += nkernels;
    if (c->prof.timing && (a = prof_event(c)) != nullptr) cudaEventRecord(a, s);
  }
  ~Timed() {
    if (!a) return;
    cudaEvent_t b = prof_event(c);
    if (!b) { c->prof.pool.push_back(a); return; }
    cudaEventRecord(b, s);
    c->prof.pending.push_back({cls, a, b});
  }
};

// Adds the elapsed times of all bracketed launches (waits for them).
void harvest(wd_ctx* c) {
  for (auto& p : c->prof.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
      c->prof.ms[p.cls] += ms;
    cudaGetLastError();
    c->prof.pool.push_back(p.a);
    c->prof.pool.push_back(p.b);
  }
  c->prof.pending.clear();
}

int check_L(int L) {
  if (L < 1 || L > WD_LMAX) {
    set_err("L = %d outside [1, %d]", L, WD_LMAX);
    return WD_EINVAL;
  }
  return WD_OK;
}

int check_ptr(const void* p, const char* name) {
  if (!p) {
    set_err("%s is NULL", name);
    return WD_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0 && is_device_ptr(p)) {
    set_err("%s is not 16-byte aligned", name);
    return WD_EINVAL;
  }
  return WD_OK;
}

// The L x L solver state, the reduction partials (one slot per block of the tall-skinny kernels,
// whose grid is a multiple of the device's SM count) and the host mirror: independent of L.
int ensure_state(wd_ctx* c) {
  CHECK(c->part.ensure((size_t)ts_max_blocks() * PART_STRIDE * sizeof(double2)));
  if (!c->st) CU(cudaMalloc(&c->st, sizeof(SolverState)));
  if (!c->bnorm2_dev) CU(cudaMalloc(&c->bnorm2_dev, 2 * WD_LMAX * sizeof(double)));
  if (!c->hm) CU(cudaMallocHost(&c->hm, sizeof(HostMirror)));
  return WD_OK;
}

int ensure_workspace(wd_ctx* c, int L) {
  if (c->L == L && c->st) return WD_OK;
  for (auto& b : c->blk) b.release();
  c->L = 0;
  const size_t bytes = block_bytes(c, L);
  for (int i = 0; i < B_CORE; ++i) CHECK(c->blk[i].ensure(bytes));
  CHECK(ensure_state(c));
  c->L = L;
  return WD_OK;
}

// Picks the low-precision sweep's tile (RHS per thread, threads per CTA, min CTAs per SM, staging) for this
// lattice, storage and L by timing every candidate on the context's blocks (zeroed first); the
// winner is kept in the context.
int autotune_lp(wd_ctx* c, int storage, int L, cudaStream_t s) {
  static const int cand[][4] = {{1, 64, 0, 0},  {1, 128, 0, 0}, {1, 256, 0, 0}, {2, 64, 0, 0},
                                {2, 128, 0, 0}, {2, 256, 0, 0}, {0, 128, 0, 0}, {2, 64, 8, 0},
                                {2, 64, 0, 1},  {1, 64, 12, 0}};
  const size_t bytes = (size_t)c->op.g.V * 12 * L * lp_elem_bytes(storage);
  void* u_lp = c->blk32[0].p;
  void* a = c->blk32[1].p;
  void* b = c->blk32[2].p;
  CU(cudaMemsetAsync(u_lp, 0, bytes, s));
  CU(cudaMemsetAsync(a, 0, bytes, s));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_i = 0;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < (int)(sizeof(cand) / sizeof(cand[0])) && err == cudaSuccess; ++i) {
    if (cand[i][0] > 0 && L % cand[i][0] != 0) continue;
    if (cand[i][3] && L % 2 != 0) continue;
    err = launch_jacobi_lp_tiled(c->op, storage, a, u_lp, b, nullptr, L, cand[i][0], cand[i][1],
                                 cand[i][2], cand[i][3], s);
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep)
      err = launch_jacobi_lp_tiled(c->op, storage, a, u_lp, b, nullptr, L, cand[i][0], cand[i][1],
                                   cand[i][2], cand[i][3], s);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms < best) { best = ms; best_i = i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CU(err);
  c->tile_r[storage][L] = cand[best_i][0];
  c->tile_block[storage][L] = cand[best_i][1];
  c->tile_minb[storage][L] = cand[best_i][2];
  c->tile_staged[storage][L] = cand[best_i][3];
  c->tile_set[storage][L] = true;
  return WD_OK;
}

// Double-float blocks take 16 bytes per complex number, like FP64 blocks.  The double-float sweep
// takes 1 or 2 RHS per thread in 128-thread CTAs, or 1 RHS in packed FP32x2 arithmetic; the
// fastest for this lattice and L is kept.
int ensure_workspace_df(wd_ctx* c, int L, cudaStream_t s) {
  const size_t bytes = (size_t)c->op.g.V * 12 * L * 16;
  for (auto& b : c->blk32) CHECK(b.ensure(bytes));
  if (c->tile_set[LP_DF][L]) return WD_OK;
  void* u_df = c->blk32[0].p;
  void* a = c->blk32[1].p;
  void* b = c->blk32[2].p;
  CU(cudaMemsetAsync(u_df, 0, bytes, s));
  CU(cudaMemsetAsync(a, 0, bytes, s));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  // (RHS per thread, packed): scalar, scalar with 2 RHS, packed FP32x2, packed with grid sums
  static const int cand[][2] = {{1, 0}, {2, 0}, {1, 1}, {1, 2}};
  float best = 1e30f;
  int best_i = 0;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < 4 && err == cudaSuccess; ++i) {
    const int r = cand[i][0], pk = cand[i][1];
    if (L % r != 0) continue;
    if (pk == 2 && !c->op.links_unitary) continue;
    err = launch_jacobi_df(c->op, a, u_df, b, nullptr, L, r, 128, pk, s);
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep)
      err = launch_jacobi_df(c->op, a, u_df, b, nullptr, L, r, 128, pk, s);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms < best) { best = ms; best_i = i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CU(err);
  c->tile_r[LP_DF][L] = cand[best_i][0];
  c->tile_block[LP_DF][L] = 128;
  c->tile_minb[LP_DF][L] = 0;
  c->tile_staged[LP_DF][L] = cand[best_i][1];
  c->tile_set[LP_DF][L] = true;
  return WD_OK;
}

int ensure_workspace_lp(wd_ctx* c, int storage, int L, cudaStream_t s) {
  const size_t bytes = (size_t)c->op.g.V * 12 * L * lp_elem_bytes(LP_F32);
  for (auto& b : c->blk32) CHECK(b.ensure(bytes));
  if (!c->tile_set[storage][L]) CHECK(autotune_lp(c, storage, L, s));
  return WD_OK;
}

// Device pointer for an input that may live on the host: copies into `stage` when needed.
int stage_input(const void* p, size_t bytes, DevBuf& stage, const double** out, bool* staged,
                cudaStream_t s) {
  if (is_device_ptr(p)) {
    *out = static_cast<const double*>(p);
    *staged = false;
    return WD_OK;
  }
  CHECK(stage.ensure(bytes));
  CU(cudaMemcpyAsync(stage.p, p, bytes, cudaMemcpyHostToDevice, s));
  *out = stage.d();
  *staged = true;
  return WD_OK;
}

// ---- domain decomposition: halo slices and sums over ranks
// Sites in one t-slice and the number of halo rows (12 per site) at each end of a block.
long long slice_sites(const wd_ctx* c) {
  return (long long)c->op.g.d[0] * c->op.g.d[1] * c->op.g.d[2];
}
constexpr int DOM_REDUCE_DOUBLES = 2 * WD_LMAX * WD_LMAX + 2 * WD_LMAX;

int dom_staging(wd_ctx* c, int L) {
  const size_t slice = (size_t)slice_sites(c) * 12 * L * 16;
  const size_t need = 4 * slice + DOM_REDUCE_DOUBLES * sizeof(double);
  if (c->dom_host_bytes >= need) return WD_OK;
  if (c->dom_host) cudaFreeHost(c->dom_host);
  c->dom_host = nullptr;
  c->dom_host_bytes = 0;
  CU(cudaMallocHost(&c->dom_host, need));
  c->dom_host_bytes = need;
  return WD_OK;
}

// Fills the two halo slices of a block (N x L, site-major, the context's extended slab) from the
// neighbouring ranks: the first and last interior slices go out, the received slices come in.
int halo_exchange(wd_ctx* c, double* blk, int L, cudaStream_t s) {
  if (!c->dom_on) return WD_OK;
  CHECK(dom_staging(c, L));
  const long long Vs = slice_sites(c), V = c->op.g.V;
  const size_t slice = (size_t)Vs * 12 * L * 16;
  const size_t per_site = (size_t)12 * L * 2;   // doubles
  char* h = static_cast<char*>(c->dom_host);
  CU(cudaMemcpyAsync(h, blk + (size_t)Vs * per_site, slice, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(h + slice, blk + (size_t)(V - 2 * Vs) * per_site, slice,
                     cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (c->dom.exchange(h, h + slice, h + 2 * slice, h + 3 * slice, slice, c->dom.user) != 0) {
    set_err("wd_domain.exchange failed");
    return WD_ECUDA;
  }
  CU(cudaMemcpyAsync(blk, h + 2 * slice, slice, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(blk + (size_t)(V - Vs) * per_site, h + 3 * slice, slice,
                     cudaMemcpyHostToDevice, s));
  return WD_OK;
}

// Sums n doubles of device memory over all ranks, in place.
int dom_sum(wd_ctx* c, void* dev, int n, cudaStream_t s) {
  if (!c->dom_on) return WD_OK;
  CHECK(dom_staging(c, 1));
  double* h = reinterpret_cast<double*>(static_cast<char*>(c->dom_host) + c->dom_host_bytes -
                                        DOM_REDUCE_DOUBLES * sizeof(double));
  CU(cudaMemcpyAsync(h, dev, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (c->dom.allreduce(h, n, c->dom.user) != 0) {
    set_err("wd_domain.allreduce failed");
    return WD_ECUDA;
  }
  CU(cudaMemcpyAsync(dev, h, n * sizeof(double), cudaMemcpyHostToDevice, s));
  return WD_OK;
}

// Rows of the reductions and block updates (the interior of a slab; all rows without a domain),
// and the offset of the first such row in doubles.
long long own_rows(const wd_ctx* c) {
  return 12LL * (c->op.g.V - (c->dom_on ? 2 * slice_sites(c) : 0));
}
size_t own_offset(const wd_ctx* c, int L) {
  return c->dom_on ? (size_t)slice_sites(c) * 12 * L * 2 : 0;
}

// G = M R with j Jacobi sweeps; `a` and `b` are two FP64 scratch blocks, the result pointer is
// returned in *res (one of a, b).  j = 0 copies R.  Modes PM_F32 and PM_BF16 run the sweeps in
// FP32 arithmetic (FP32 links and A_D^{-1}) on blocks stored in FP32 or BF16 and write the last
// sweep to `a` in FP64.
int precondition(wd_ctx* c, const double* R, double* a, double* b, double** res, int L, int j,
                 int mode, long long* hop_count, cudaStream_t s) {
  const Op& op = c->op;
  if (j == 0 && mode != PM_NET) {
    LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(a, R, block_bytes(c, L), cudaMemcpyDeviceToDevice, s));
    *res = a;
    return WD_OK;
  }
  if (mode == PM_NET) {   // learned network
    *res = a;
    Timed timed_(c, WD_K_NET, 0, s);
    CHECK(wd_net_precondition(c, c->active_net, R, a, L, c->net_bf16, s));
    return WD_OK;
  }
  if (mode == PM_DF) {
    *res = a;
    if (j == 1) {
      LAUNCH(WD_K_SITE_INV, 1, launch_site_inverse_df(op, R, nullptr, nullptr, a, L, s));
      return WD_OK;
    }
    CHECK(ensure_workspace_df(c, L, s));
    void* u_df = c->blk32[0].p;
    void* cur = c->blk32[1].p;
    void* nxt = c->blk32[2].p;
    LAUNCH(WD_K_SITE_INV, 1, launch_site_inverse_df(op, R, u_df, cur, nullptr, L, s));
    for (int i = 1; i < j; ++i) {
      const bool last = i == j - 1;
      LAUNCH(WD_K_JACOBI_LP, 1,
             launch_jacobi_df(op, cur, u_df, last ? nullptr : nxt, last ? a : nullptr, L,
                              c->tile_r[LP_DF][L], c->tile_block[LP_DF][L],
                              c->tile_staged[LP_DF][L], s));
      if (hop_count) ++*hop_count;
      void* t = cur;
      cur = nxt;
      nxt = t;
    }
    return WD_OK;
  }
  if (mode == PM_F32 || mode == PM_BF16) {
    const int st = lp_storage(mode);
    *res = a;
    if (j == 1) {
      LAUNCH(WD_K_SITE_INV, 1, launch_site_inverse_lp(op, st, R, nullptr, nullptr, a, L, s));
      return WD_OK;
    }
    CHECK(ensure_workspace_lp(c, st, L, s));
    void* u_lp = c->blk32[0].p;
    void* cur = c->blk32[1].p;
    void* nxt = c->blk32[2].p;
    LAUNCH(WD_K_SITE_INV, 1, launch_site_inverse_lp(op, st, R, u_lp, cur, nullptr, L, s));
    for (int i = 1; i < j; ++i) {
      const bool last = i == j - 1;
      LAUNCH(WD_K_JACOBI_LP, 1,
             launch_jacobi_lp_tiled(op, st, cur, u_lp, last ? nullptr : nxt, last ? a : nullptr,
                                    L, c->tile_r[st][L], c->tile_block[st][L],
                                    c->tile_minb[st][L], c->tile_staged[st][L], s));
      if (hop_count) ++*hop_count;
      void* t = cur;
      cur = nxt;
      nxt = t;
    }
    return WD_OK;
  }
  LAUNCH(WD_K_SITE_INV, 1, launch_site_inverse_f64(op, R, a, L, s));
  double* cur = a;
  double* nxt = b;
  for (int i = 1; i < j; ++i) {
    CHECK(halo_exchange(c, cur, L, s));
    LAUNCH(WD_K_JACOBI, stencil_kernels(op), launch_jacobi_f64(op, cur, R, nxt, L, s));
    if (hop_count) ++*hop_count;
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  *res = cur;
  return WD_OK;
}

int read_back(wd_ctx* c, cudaStream_t s) {
  CU(cudaMemcpyAsync(c->hm, reinterpret_cast<char*>(c->st) + offsetof(SolverState, rnorm2),
                     sizeof(double) * WD_LMAX, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(&c->hm->status, reinterpret_cast<char*>(c->st) + offsetof(SolverState, status),
                     sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return WD_OK;
}

constexpr int RUN_STALLED = 100;   // internal: the FP32-preconditioned run stopped improving

struct RunResult {
  int status;
  int k;
  double rec[WD_LMAX];
};

double max_rel(const double* n2, const double* b2, int L, double* rel) {
  double m = 0.0;
  for (int i = 0; i < L; ++i) {
    const double r = std::sqrt(n2[i]) / std::sqrt(b2[i]);
    if (rel) rel[i] = r;
    if (!(r <= m)) m = r;   // NaN propagates
  }
  return m;
}

// One run of preconditioned block BiCGGR from the current X (Sec. 2, algorithm box).
int run_bbicggr(wd_ctx* c, const double* B, double* X, int L, int j, int precision, bool df,
                double tol, int maxit, double div_thresh, const double* b2, bbicggr_opts* o, int* hist_n,
                long long* hop_count, RunResult* out, cudaStream_t s) {
  const Op& op = c->op;
  const long long rows = own_rows(c);        // the rows this context owns (its slab's interior)
  const size_t off = own_offset(c, L);
  auto in = [off](double* p) { return p + off; };
  auto cin = [off](const double* p) { return p + off; };
  const size_t bytes = block_bytes(c, L);
  double* R = c->blk[B_R].d();
  double* P = c->blk[B_P].d();
  double* V = c->blk[B_V].d();
  double* W = c->blk[B_W].d();
  double* U = c->blk[B_U].d();
  double* Y = c->blk[B_Y].d();
  double* Rt = c->blk[B_RT].d();
  double* pF = c->blk[B_F].d();
  double* pG = c->blk[B_G].d();
  double* pT = c->blk[B_T].d();
  double2* part = static_cast<double2*>(c->part.p);
  SolverState* st = c->st;
  CU(cudaMemsetAsync(&st->status, 0, sizeof(int), s));

  // R_0 = B - A X_0;  P_0 = R_0;  R~_0 = R_0
  CHECK(halo_exchange(c, X, L, s));
  LAUNCH(WD_K_RESID, stencil_kernels(op), launch_resid_f64(op, X, B, R, L, s));
  ++*hop_count;
  LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(P, R, bytes, cudaMemcpyDeviceToDevice, s));
  LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(Rt, R, bytes, cudaMemcpyDeviceToDevice, s));
  LAUNCH(WD_K_GRAM, 2, launch_gram(in(Rt), in(R), L, rows, part, st, GRAM_RTR, true, s));
  CHECK(dom_sum(c, st->rtr, 2 * L * L, s));
  CHECK(dom_sum(c, st->rnorm2, L, s));
  CHECK(read_back(c, s));
  double m = max_rel(c->hm->rnorm2, b2, L, out->rec);
  out->k = 0;
  if (o->history && *hist_n < o->history_len) o->history[(*hist_n)++] = m;
  if (m <= tol) { out->status = WD_OK; return WD_OK; }
  if (!std::isfinite(m)) { out->status = WD_BREAKDOWN; return WD_OK; }

  // F_0 = M R_0;  V_0 = W_0 = A F_0
  double* res;
  CHECK(precondition(c, R, pF, pT, &res, L, j, precision, hop_count, s));
  if (res != pF) { pT = pF; pF = res; }
  CHECK(halo_exchange(c, pF, L, s));
  LAUNCH(WD_K_APPLY, stencil_kernels(op), launch_apply_f64(op, pF, W, L, s));
  ++*hop_count;
  LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(V, W, bytes, cudaMemcpyDeviceToDevice, s));
  LAUNCH(WD_K_TRACE, 2, launch_traces(in(W), in(R), L, rows, part, st, s));
  CHECK(dom_sum(c, &st->trwr, 3, s));
  LAUNCH(WD_K_GRAM, 2, launch_gram(in(Rt), in(V), L, rows, part, st, GRAM_RTV, false, s));
  CHECK(dom_sum(c, st->rtv, 2 * L * L, s));

  int k = 0;
  double best = m;
  int k_best = 0;
  const int stall = precision != 0 ? o->stall_window : 0;
  for (;;) {
    if (k >= maxit) { out->status = WD_NOT_CONVERGED; break; }
    LAUNCH(WD_K_SOLVE_LL, 1, launch_solve_alpha(st, L, s));                       // alpha_k, zeta_k
    LAUNCH(WD_K_UPDATE_U, 1, launch_update_u(in(P), in(V), in(U), L, rows, st, s, df));           // U_k = (P_k - zeta_k V_k) alpha_k
    CHECK(precondition(c, U, pG, pT, &res, L, j, precision, hop_count, s));   // G_k = M U_k
    if (res != pG) { pT = pG; pG = res; }
    CHECK(halo_exchange(c, pG, L, s));
    LAUNCH(WD_K_APPLY, stencil_kernels(op), launch_apply_f64(op, pG, Y, L, s));                  // Y_k = A G_k
    ++*hop_count;
    LAUNCH(WD_K_UPDATE_XR, 2, launch_update_xr(in(X), cin(pF), cin(pG), in(R), cin(W), cin(Y), cin(Rt), L, rows, part, st, s, df));   // X_{k+1}, R_{k+1}
    CHECK(dom_sum(c, st->rtr_new, 2 * L * L, s));
    CHECK(dom_sum(c, st->rnorm2, L, s));
    CHECK(read_back(c, s));
    if (c->hm->status != ST_OK) { out->status = WD_BREAKDOWN; break; }
    ++k;
    m = max_rel(c->hm->rnorm2, b2, L, out->rec);
    if (o->history && *hist_n < o->history_len) o->history[(*hist_n)++] = m;
    if (!std::isfinite(m)) { out->status = WD_BREAKDOWN; break; }
    if (m <= tol) { out->status = WD_OK; break; }
    if (m > div_thresh) { out->status = WD_DIVERGED; break; }
    if (m < best) { best = m; k_best = k; }
    if (stall > 0 && k - k_best >= stall) { out->status = RUN_STALLED; break; }
    CHECK(precondition(c, R, pF, pT, &res, L, j, precision, hop_count, s));   // F_{k+1} = M R_{k+1}
    if (res != pF) { pT = pF; pF = res; }
    CHECK(halo_exchange(c, pF, L, s));
    LAUNCH(WD_K_APPLY, stencil_kernels(op), launch_apply_f64(op, pF, W, L, s));                  // W_{k+1} = A F_{k+1}
    ++*hop_count;
    LAUNCH(WD_K_TRACE, 2, launch_traces(in(W), in(R), L, rows, part, st, s));  // Tr[W^H R], Tr[W^H W]
    CHECK(dom_sum(c, &st->trwr, 3, s));
    LAUNCH(WD_K_SOLVE_LL, 1, launch_solve_gamma(st, L, s));                       // gamma_k
    LAUNCH(WD_K_UPDATE_PV, 2, launch_update_pv(in(P), in(V), cin(R), cin(W), cin(U), cin(Y), cin(Rt), L, rows, part, st, s, df));   // P_{k+1}, V_{k+1}
    CHECK(dom_sum(c, st->rtv, 2 * L * L, s));
  }
  out->k = k;
  return WD_OK;
}


}  // namespace

const Op* wd_ctx_op(const wd_ctx* c) { return &c->op; }
int wd_ctx_device(const wd_ctx* c) { return c->device; }
void wd_ctx_count_launches(wd_ctx* c, int cls, int nkernels) {
  if (cls >= 0 && cls < WD_K_COUNT) c->prof.kernels[cls] += nkernels;
}

void wd_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" {

void bbicggr_default_opts(bbicggr_opts* o) {
  if (!o) return;
  o->maxit = 10000;
  o->div_thresh = 1e2;
  o->max_restarts = 3;
  o->precision = 0;
  o->history = nullptr;
  o->history_len = 0;
  o->stall_window = 16;
  o->net = nullptr;
}

const char* wd_strerror(int code) {
  switch (code) {
    case WD_OK: return "WD_OK";
    case WD_EINVAL: return "WD_EINVAL";
    case WD_ENOMEM: return "WD_ENOMEM";
    case WD_ECUDA: return "WD_ECUDA";
    case WD_NOT_CONVERGED: return "WD_NOT_CONVERGED";
    case WD_DIVERGED: return "WD_DIVERGED";
    case WD_BREAKDOWN: return "WD_BREAKDOWN";
    default: return "WD_UNKNOWN";
  }
}

const char* wd_last_error(void) { return g_err; }

void wd_destroy(wd_ctx* c) {
  if (!c) return;
  harvest(c);
  for (auto e : c->prof.pool) cudaEventDestroy(e);
  cudaFree(c->op.links);
  cudaFree(c->op.clov);
  cudaFree(c->op.clov_inv);
  cudaFree(c->op.links32);
  cudaFree(c->op.clov_inv32);
  cudaFree(c->op.clov_bound32);
  cudaFree(c->op.links32s);
  cudaFree(c->op.clov_inv32s);
  cudaFree(c->op.links_x3);
  cudaFree(c->op.xexp);
  for (auto& b : c->blk) b.release();
  for (auto& b : c->blk32) b.release();
  c->part.release();
  c->stage_in.release();
  c->stage_out.release();
  cudaFree(c->st);
  cudaFree(c->bnorm2_dev);
  cudaFree(c->gctl);
  cudaFree(c->ghist);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  cudaFreeHost(c->hm);
  if (c->dom_host) cudaFreeHost(c->dom_host);
  delete c;
}

static int create_impl(wd_ctx* c, const void* links, const int dims[4], cudaStream_t s) {
  Op& op = c->op;
  const size_t V = op.g.V;
  const size_t lbytes = V * 4 * 18 * sizeof(double);
  CU(cudaMalloc(&op.links, lbytes));
  CU(cudaMalloc(&op.clov, V * 2 * CLOV_REALS * sizeof(double)));
  CU(cudaMalloc(&op.clov_inv, V * 2 * CLOV_REALS * sizeof(double)));
  CU(cudaMalloc(&op.links32, V * 4 * 18 * sizeof(float)));
  CU(cudaMalloc(&op.clov_inv32, V * 2 * CLOV_REALS * sizeof(float)));
  CU(cudaMalloc(&op.clov_bound32, V * 2 * sizeof(float)));
  CU(cudaMalloc(&op.links32s, V * 4 * 5 * sizeof(float4)));
  CU(cudaMalloc(&op.clov_inv32s, V * 2 * (CLOV_REALS / 4) * sizeof(float4)));
  CU(cudaMemcpyAsync(op.links, links, lbytes, cudaMemcpyDefault, s));
  // [0]: a singular A_D block; [1]: a link that is not special unitary; [2]: a link with a row or
  // column of norm above 1
  int* flag;
  CU(cudaMalloc(&flag, 3 * sizeof(int)));
  CU(cudaMemsetAsync(flag, 0, 3 * sizeof(int), s));
  CU(launch_clover_build(op, flag, s));
  CU(launch_lp_operator_copies(op, flag + 1, s));
  int h[3] = {0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(h, flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(flag);
  CU(e);
  c->links_su3 = h[1] == 0;
  op.link12 = c->links_su3 ? 1 : 0;
  op.links_unitary = h[2] == 0 ? 1 : 0;
  if (h[0]) {
    set_err("a 6x6 clover block A_D is singular for kappa=%g c_SW=%g", op.kappa, op.csw);
    return WD_BREAKDOWN;
  }
  if (op.links_unitary) {   // the FP32-lane form of the FP64 stencil (its bounds need unitary links)
    CU(cudaMalloc(&op.links_x3, V * 4 * 27 * sizeof(float4)));
    CU(cudaMalloc(&op.xexp, V * WD_LMAX * sizeof(int)));
    CU(launch_link_split(op, s));
    CU(cudaStreamSynchronize(s));
    op.apply_form = 1;
  }
  return WD_OK;
}

int wd_create(wd_ctx** out, const void* links, const int dims[4], double kappa, double csw,
              void* stream) {
  if (!out) { set_err("out is NULL"); return WD_EINVAL; }
  *out = nullptr;
  if (!links || !dims) { set_err("links or dims is NULL"); return WD_EINVAL; }
  long long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2 || dims[m] > 4096) {
      set_err("dims[%d] = %d outside [2, 4096]", m, dims[m]);
      return WD_EINVAL;
    }
    V *= dims[m];
  }
  if (V > (1LL << 26)) { set_err("volume %lld above 2^26 sites", V); return WD_EINVAL; }
  if (!std::isfinite(kappa) || !std::isfinite(csw)) { set_err("kappa or c_SW not finite"); return WD_EINVAL; }
  if (reinterpret_cast<uintptr_t>(links) % 16 != 0 && is_device_ptr(links)) {
    set_err("links not 16-byte aligned");
    return WD_EINVAL;
  }
  wd_ctx* c = new (std::nothrow) wd_ctx();
  if (!c) { set_err("host allocation failed"); return WD_ENOMEM; }
  cudaGetDevice(&c->device);
  // The static scratch array of jacobi_precond_noalloc is loaded on this device now, so that it
  // is never allocated later inside an allocation-free call.
  int rc0 = noalloc_reserve();
  if (rc0 != WD_OK) { delete c; return rc0; }
  c->op.g = make_geom(dims);
  c->op.kappa = kappa;
  c->op.csw = csw;
  int rc = create_impl(c, links, dims, static_cast<cudaStream_t>(stream));
  if (rc != WD_OK) { wd_destroy(c); return rc; }
  *out = c;
  return WD_OK;
}

int wd_profile_enable(wd_ctx* c, int timing_on) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  harvest(c);
  c->prof.timing = timing_on != 0;
  return WD_OK;
}

int wd_profile_reset(wd_ctx* c) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  harvest(c);
  for (int i = 0; i < WD_K_COUNT; ++i) { c->prof.kernels[i] = 0; c->prof.ms[i] = 0.0; }
  return WD_OK;
}

int wd_profile_read(const wd_ctx* c, int cls, long long* launches, double* ms) {
  if (!c || cls < 0 || cls >= WD_K_COUNT) { set_err("bad context or kernel class"); return WD_EINVAL; }
  if (launches) *launches = c->prof.kernels[cls];
  if (ms) *ms = c->prof.ms[cls];
  return WD_OK;
}

const char* wd_profile_name(int cls) {
  static const char* names[WD_K_COUNT] = {
      "dslash_apply", "dslash_resid", "dslash_jacobi", "site_inverse", "update_u", "update_xr",
      "update_pv", "gram", "trace", "solve_ll", "colnorm", "copy", "convert", "net",
      "dslash_jacobi_lp"};
  return (cls >= 0 && cls < WD_K_COUNT) ? names[cls] : "unknown";
}

static int tile_storage(int precision, int* storage) {
  if (precision == 1) { *storage = LP_F32; return WD_OK; }
  if (precision == 3) { *storage = LP_BF16; return WD_OK; }
  if (precision == 4) { *storage = LP_DF; return WD_OK; }
  set_err("precision %d has no sweep tile (1 = FP32, 3 = BF16 storage, 4 = double-float)", precision);
  return WD_EINVAL;
}

int wd_set_tile(wd_ctx* c, int L, int precision, int rhs_per_thread, int block, int min_blocks,
                int staged) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  CHECK(check_L(L));
  int st;
  CHECK(tile_storage(precision, &st));
  if (st == LP_DF) {   // 1 or 2 RHS per thread, 128 threads; staged 1 = packed, 2 = packed with
                       // grid sums (1 RHS; unitary links)
    if ((rhs_per_thread != 1 && rhs_per_thread != 2) || L % rhs_per_thread != 0 || block != 128 ||
        min_blocks != 0 || staged < 0 || staged > 2 || (staged != 0 && rhs_per_thread != 1) ||
        (staged == 2 && !c->op.links_unitary)) {
      set_err("double-float tile (%d RHS/thread, %d threads) not available for L = %d",
              rhs_per_thread, block, L);
      return WD_EINVAL;
    }
    c->tile_r[st][L] = rhs_per_thread;
    c->tile_block[st][L] = block;
    c->tile_minb[st][L] = 0;
    c->tile_staged[st][L] = staged;
    c->tile_set[st][L] = true;
    return WD_OK;
  }
  const bool split = rhs_per_thread == 0 && block == 128 && min_blocks == 0;
  const bool capped = block == 64 && ((min_blocks == 8 && rhs_per_thread != 0) ||
                                      (min_blocks == 12 && rhs_per_thread == 1));
  const bool pipe = staged == 1 && rhs_per_thread == 2 && block == 64 && min_blocks == 0 && L % 2 == 0;
  if ((staged != 0 && !pipe) ||
      (!staged && !split && ((rhs_per_thread != 1 && rhs_per_thread != 2) || L % rhs_per_thread != 0 ||
                             (block != 64 && block != 128 && block != 256) ||
                             (min_blocks != 0 && !capped)))) {
    set_err("tile (%d RHS/thread, %d threads, min %d blocks, staged %d) not available for L = %d",
            rhs_per_thread, block, min_blocks, staged, L);
    return WD_EINVAL;
  }
  c->tile_r[st][L] = rhs_per_thread;
  c->tile_block[st][L] = block;
  c->tile_minb[st][L] = min_blocks;
  c->tile_staged[st][L] = staged;
  c->tile_set[st][L] = true;
  return WD_OK;
}

int wd_tuned_tile(const wd_ctx* c, int L, int precision, int* rhs_per_thread, int* block,
                  int* min_blocks, int* staged) {
  int st;
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  CHECK(tile_storage(precision, &st));
  if (L < 1 || L > WD_LMAX || !c->tile_set[st][L]) { set_err("no tuned tile for this L"); return WD_EINVAL; }
  if (rhs_per_thread) *rhs_per_thread = c->tile_r[st][L];
  if (block) *block = c->tile_block[st][L];
  if (min_blocks) *min_blocks = c->tile_minb[st][L];
  if (staged) *staged = c->tile_staged[st][L];
  return WD_OK;
}

int wd_link_reals(const wd_ctx* c, int* reals) {
  if (!c || !reals) { set_err("ctx or reals is NULL"); return WD_EINVAL; }
  *reals = c->op.link12 ? 12 : 18;
  return WD_OK;
}

int wd_set_link_reals(wd_ctx* c, int reals) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  if (reals != 12 && reals != 18) { set_err("link format %d not in {12, 18}", reals); return WD_EINVAL; }
  if (reals == 12 && !c->links_su3) {
    set_err("the links are not special unitary to %g: their third rows cannot be rebuilt", LINK12_TOL);
    return WD_EINVAL;
  }
  c->op.link12 = reals == 12 ? 1 : 0;
  return WD_OK;
}

int wd_set_apply_form(wd_ctx* c, int form) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  if (form != 0 && form != 1) { set_err("stencil form %d not in {0, 1}", form); return WD_EINVAL; }
  if (form == 1 && !c->op.links_x3) {
    set_err("the FP32-lane stencil needs links whose rows and columns have norm <= 1 + %g", LINK12_TOL);
    return WD_EINVAL;
  }
  c->op.apply_form = form;
  return WD_OK;
}

int wd_get_apply_form(const wd_ctx* c) { return c ? c->op.apply_form : -1; }

int wd_set_domain(wd_ctx* c, const wd_domain* dom) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  if (!dom) { c->dom_on = false; return WD_OK; }
  if (!dom->exchange || !dom->allreduce) { set_err("wd_domain needs exchange and allreduce"); return WD_EINVAL; }
  if (c->op.g.d[3] < 3) {
    set_err("a domain's slab needs Lt >= 3 (one interior slice and a halo slice on each side)");
    return WD_EINVAL;
  }
  c->dom = *dom;
  c->dom_on = true;
  return WD_OK;
}

int wd_query(const wd_ctx* c, int dims[4], long long* volume, double* kappa, double* csw) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  if (dims) for (int m = 0; m < 4; ++m) dims[m] = c->op.g.d[m];
  if (volume) *volume = c->op.g.V;
  if (kappa) *kappa = c->op.kappa;
  if (csw) *csw = c->op.csw;
  return WD_OK;
}

int wd_apply(wd_ctx* c, const void* X, void* Y, int L, void* stream) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  CHECK(check_L(L));
  CHECK(check_ptr(X, "X"));
  CHECK(check_ptr(Y, "Y"));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = block_bytes(c, L);
  const double* xd;
  bool staged_x;
  CHECK(stage_input(X, bytes, c->stage_in, &xd, &staged_x, s));
  const bool y_dev = is_device_ptr(Y);
  double* yd = static_cast<double*>(Y);
  if (!y_dev) { CHECK(c->stage_out.ensure(bytes)); yd = c->stage_out.d(); }
  if (c->dom_on) {   // refresh the halo slices of a copy of X (the caller's X is not written)
    CHECK(c->stage_in.ensure(bytes));
    if (xd != c->stage_in.d())
      LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(c->stage_in.d(), xd, bytes, cudaMemcpyDeviceToDevice, s));
    xd = c->stage_in.d();
    CHECK(halo_exchange(c, c->stage_in.d(), L, s));
  }
  LAUNCH(WD_K_APPLY, stencil_kernels(c->op), launch_apply_f64(c->op, xd, yd, L, s));
  if (!y_dev) CU(cudaMemcpyAsync(Y, yd, bytes, cudaMemcpyDeviceToHost, s));
  if (staged_x || !y_dev) CU(cudaStreamSynchronize(s));
  harvest(c);
  return WD_OK;
}

int jacobi_precond(wd_ctx* c, const void* R, void* G, int L, int j, int precision, void* stream) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  CHECK(check_L(L));
  CHECK(check_ptr(R, "R"));
  CHECK(check_ptr(G, "G"));
  if (j < 0) { set_err("j = %d < 0", j); return WD_EINVAL; }
  if (precision != PM_F64 && precision != PM_F32 && precision != PM_BF16 && precision != PM_DF) {
    set_err("precision %d not in {0, 1, 3, 4}", precision);
    return WD_EINVAL;
  }
  if (c->dom_on && precision != PM_F64) {
    set_err("with a domain set, the Jacobi preconditioner runs FP64 sweeps (precision 0)");
    return WD_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = block_bytes(c, L);
  const double* rd;
  bool staged_r;
  CHECK(stage_input(R, bytes, c->stage_in, &rd, &staged_r, s));
  const bool g_dev = is_device_ptr(G);
  double* gd = static_cast<double*>(G);
  if (!g_dev) { CHECK(c->stage_out.ensure(bytes)); gd = c->stage_out.d(); }
  // ping-pong between the output and one workspace block
  CHECK(ensure_workspace(c, L));
  double* tmp = c->blk[B_T].d();
  double* res;
  // Arrange the sweeps so that the last one lands in gd: with j sweeps the result sits in the
  // first buffer when j is odd.
  double* first = (j % 2 == 1) ? gd : tmp;
  double* second = (j % 2 == 1) ? tmp : gd;
  if (precision != PM_F64) { first = gd; second = tmp; }   // low-precision sweeps finish in `first`
  CHECK(precondition(c, rd, first, second, &res, L, j, precision, nullptr, s));
  if (res != gd) LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(gd, res, bytes, cudaMemcpyDeviceToDevice, s));
  if (!g_dev) CU(cudaMemcpyAsync(G, gd, bytes, cudaMemcpyDeviceToHost, s));
  if (staged_r || !g_dev) CU(cudaStreamSynchronize(s));
  harvest(c);
  return WD_OK;
}

// ---- block updates of one outer iteration on caller-supplied device blocks
namespace {
int check_update_args(wd_ctx* c, int L, int precision, std::initializer_list<const void*> blocks) {
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  CHECK(check_L(L));
  if (precision != 0 && precision != 1) {
    set_err("precision %d not in {0 (FP64), 1 (double-float)}", precision);
    return WD_EINVAL;
  }
  for (const void* p : blocks) {
    CHECK(check_ptr(p, "block"));
    if (!is_device_ptr(p)) { set_err("the block updates take device buffers only"); return WD_EINVAL; }
  }
  return ensure_state(c);
}

// Host L x L complex128 coefficients (row-major) into the device solver state.
int put_coef(wd_ctx* c, double2* dst, const void* host, int L, cudaStream_t s) {
  if (!host) { set_err("coefficient matrix is NULL"); return WD_EINVAL; }
  const double2* h = static_cast<const double2*>(host);
  CU(cudaMemcpyAsync(dst, h, sizeof(double2) * L * L, cudaMemcpyHostToDevice, s));
  return WD_OK;
}

int put_zeta(wd_ctx* c, const double* zeta, cudaStream_t s) {
  if (!zeta) { set_err("zeta is NULL"); return WD_EINVAL; }
  CU(cudaMemcpyAsync(&c->st->zeta, zeta, sizeof(double2), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(&c->st->status, 0, sizeof(int), s));
  return WD_OK;
}
}  // namespace

int bb_update_u(wd_ctx* c, const void* P, const void* V, void* U, int L, const double* zeta,
                const void* alpha, int precision, void* stream) {
  CHECK(check_update_args(c, L, precision, {P, V, U}));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long rows = (long long)c->op.g.V * 12;
  CHECK(put_zeta(c, zeta, s));
  CHECK(put_coef(c, c->st->alpha, alpha, L, s));
  LAUNCH(WD_K_UPDATE_U, 1,
         launch_update_u(static_cast<const double*>(P), static_cast<const double*>(V),
                         static_cast<double*>(U), L, rows, c->st, s, precision == 1));
  CU(cudaStreamSynchronize(s));
  harvest(c);
  return WD_OK;
}

int bb_update_xr(wd_ctx* c, void* X, const void* F, const void* G, void* R, const void* W,
                 const void* Y, const void* Rt, int L, const double* zeta, void* rtr_new,
                 double* rnorm2, int precision, void* stream) {
  CHECK(check_update_args(c, L, precision, {X, F, G, R, W, Y, Rt}));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long rows = (long long)c->op.g.V * 12;
  CHECK(put_zeta(c, zeta, s));
  LAUNCH(WD_K_UPDATE_XR, 2,
         launch_update_xr(static_cast<double*>(X), static_cast<const double*>(F),
                          static_cast<const double*>(G), static_cast<double*>(R),
                          static_cast<const double*>(W), static_cast<const double*>(Y),
                          static_cast<const double*>(Rt), L, rows,
                          static_cast<double2*>(c->part.p), c->st, s, precision == 1));
  SolverState h;
  CU(cudaMemcpyAsync(&h, c->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  harvest(c);
  if (rtr_new) std::memcpy(rtr_new, h.rtr_new, sizeof(double2) * L * L);
  if (rnorm2) std::memcpy(rnorm2, h.rnorm2, sizeof(double) * L);
  return WD_OK;
}

int bb_update_pv(wd_ctx* c, void* P, void* V, const void* R, const void* W, const void* U,
                 const void* Y, const void* Rt, int L, const void* gamma, void* rtv,
                 int precision, void* stream) {
  CHECK(check_update_args(c, L, precision, {P, V, R, W, U, Y, Rt}));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long rows = (long long)c->op.g.V * 12;
  CU(cudaMemsetAsync(&c->st->status, 0, sizeof(int), s));
  CHECK(put_coef(c, c->st->gamma, gamma, L, s));
  LAUNCH(WD_K_UPDATE_PV, 2,
         launch_update_pv(static_cast<double*>(P), static_cast<double*>(V),
                          static_cast<const double*>(R), static_cast<const double*>(W),
                          static_cast<const double*>(U), static_cast<const double*>(Y),
                          static_cast<const double*>(Rt), L, rows,
                          static_cast<double2*>(c->part.p), c->st, s, precision == 1));
  SolverState h;
  CU(cudaMemcpyAsync(&h, c->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  harvest(c);
  if (rtv) std::memcpy(rtv, h.rtv, sizeof(double2) * L * L);
  return WD_OK;
}

int bbicggr_solve(wd_ctx* c, const void* B, void* X, int L, int j, double tol,
                  const bbicggr_opts* opts, bbicggr_info* info, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!c) { set_err("ctx is NULL"); return WD_EINVAL; }
  CHECK(check_L(L));
  CHECK(check_ptr(B, "B"));
  CHECK(check_ptr(X, "X"));
  if (j < 0) { set_err("j = %d < 0", j); return WD_EINVAL; }
  if (!(tol > 0.0)) { set_err("tol must be > 0"); return WD_EINVAL; }
  bbicggr_opts o;
  bbicggr_default_opts(&o);
  if (opts) o = *opts;
  if (o.maxit < 0 || o.max_restarts < 0 || !(o.div_thresh > 0.0) || o.stall_window < 0) {
    set_err("invalid options");
    return WD_EINVAL;
  }
  if (o.precision < 0 || o.precision > 5) { set_err("precision %d not in {0, ..., 5}", o.precision); return WD_EINVAL; }
  if (c->dom_on && (o.precision != 0 || o.net)) {
    set_err("a domain-decomposed solve takes the FP64 Jacobi preconditioner (precision 0)");
    return WD_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CHECK(ensure_workspace(c, L));
  const size_t bytes = block_bytes(c, L);
  const long long rows = own_rows(c);
  const size_t off = own_offset(c, L);

  const double* Bd = static_cast<const double*>(B);
  if (!is_device_ptr(B)) {
    CHECK(c->blk[B_B].ensure(bytes));
    CU(cudaMemcpyAsync(c->blk[B_B].d(), B, bytes, cudaMemcpyHostToDevice, s));
    Bd = c->blk[B_B].d();
  }
  const bool x_dev = is_device_ptr(X);
  double* Xd = static_cast<double*>(X);
  if (!x_dev) {
    CHECK(c->blk[B_XS].ensure(bytes));
    Xd = c->blk[B_XS].d();
    CU(cudaMemcpyAsync(Xd, X, bytes, cudaMemcpyHostToDevice, s));
  }
  double b2[WD_LMAX];
  LAUNCH(WD_K_COLNORM, 2, launch_colnorms(Bd + off, L, rows, static_cast<double2*>(c->part.p), c->bnorm2_dev, s));
  CHECK(dom_sum(c, c->bnorm2_dev, L, s));
  CU(cudaMemcpyAsync(b2, c->bnorm2_dev, L * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  for (int i = 0; i < L; ++i)
    if (!(b2[i] > 0.0) || !std::isfinite(b2[i])) {
      set_err("column %d of B is zero or not finite", i);
      return WD_EINVAL;
    }

  int status = WD_OK, iters = 0, restarts = 0, hist_n = 0, fallbacks = 0;
  int prec = precond_mode(o);
  bool df = o.precision == 2 || o.precision == 5;
  c->active_net = o.net;
  c->net_bf16 = o.net && o.precision == 3;
  const bool may_fall_back = prec != 0 && o.stall_window > 0;
  if (may_fall_back) CHECK(c->blk[B_X0].ensure(bytes));
  if (may_fall_back)   // keep X_0 for a restart with the FP64 preconditioner
    LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(c->blk[B_X0].d(), Xd, bytes, cudaMemcpyDeviceToDevice, s));
  long long mvm_paper = 0, hops = 0;
  RunResult rr{};
  double true_rel[WD_LMAX];
  double mtrue = 0.0;
  for (;;) {
    long long hop_run = 0;
    CHECK(run_bbicggr(c, Bd, Xd, L, j, prec, df, tol, o.maxit - iters, o.div_thresh, b2, &o, &hist_n,
                      &hop_run, &rr, s));
    iters += rr.k;
    hops += hop_run;
    mvm_paper += (long long)L * (2LL * ((prec == 2 ? 0 : j) + 1) * rr.k + 1);
    if (prec != 0 && may_fall_back &&
        (rr.status == RUN_STALLED || rr.status == WD_BREAKDOWN || rr.status == WD_DIVERGED) &&
        iters < o.maxit) {
      // Start over from X_0 with the FP64 preconditioner.  Restarting from the stalled iterate is
      // not used: near the critical kappa its residual lies in the operator's low-mode space, from
      // which block BiCGGR (with R~_0 = R_0 or the original R~_0) itself fails to converge.
      LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(Xd, c->blk[B_X0].d(), bytes, cudaMemcpyDeviceToDevice, s));
      prec = 0;
      df = false;
      ++fallbacks;
      continue;
    }
    if (rr.status == RUN_STALLED) rr.status = WD_NOT_CONVERGED;
    // true residual ||b_i - A x_i|| / ||b_i||
    double* T = c->blk[B_T].d();
    CHECK(halo_exchange(c, Xd, L, s));
    LAUNCH(WD_K_RESID, stencil_kernels(c->op), launch_resid_f64(c->op, Xd, Bd, T, L, s));
    ++hops;
    double t2[WD_LMAX];
    LAUNCH(WD_K_COLNORM, 2, launch_colnorms(T + off, L, rows, static_cast<double2*>(c->part.p), c->bnorm2_dev + WD_LMAX, s));
    CHECK(dom_sum(c, c->bnorm2_dev + WD_LMAX, L, s));
    CU(cudaMemcpyAsync(t2, c->bnorm2_dev + WD_LMAX, L * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    mtrue = max_rel(t2, b2, L, true_rel);
    status = rr.status;
    if (status != WD_OK) break;
    if (mtrue <= tol) break;
    if (restarts >= o.max_restarts || iters >= o.maxit) { status = WD_NOT_CONVERGED; break; }
    ++restarts;
  }
  if (!x_dev) {
    CU(cudaMemcpyAsync(X, Xd, bytes, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
  }
  c->solved_L = L;
  if (info) {
    info->status = status;
    info->iters = iters;
    info->restarts = restarts;
    info->mvm_paper = mvm_paper;
    info->mvm_actual = hops * L;
    double mr = 0.0;
    for (int i = 0; i < L; ++i) mr = (rr.rec[i] > mr || std::isnan(rr.rec[i])) ? rr.rec[i] : mr;
    info->max_rec_resid = mr;
    info->max_true_resid = mtrue;
    if (info->rec_resid) std::memcpy(info->rec_resid, rr.rec, L * sizeof(double));
    if (info->true_resid) std::memcpy(info->true_resid, true_rel, L * sizeof(double));
    info->history_count = hist_n;
    info->fallbacks = fallbacks;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  harvest(c);
  if (status != WD_OK)
    set_err("bbicggr_solve: %s after %d iterations (max recursive residual %.3e, true %.3e)",
            wd_strerror(status), iters, info ? info->max_rec_resid : 0.0, mtrue);
  return status;
}

}  // extern "C"

// ================================================================== device-controlled solves
// bbicggr_solve_batch: every job's solve becomes one branch of a single CUDA graph, with the whole
// control flow of bbicggr_solve on the device:
//   WHILE (phase)                                   one run of block BiCGGR per pass
//     IF (mode 0) run with the job's preconditioner
//     IF (mode 1) run with the FP64 Jacobi preconditioner (after a fallback; X restored to X_0)
//     true residual; phase check: fall back, restart from X, or stop
//   run = R_0, F_0, W_0 ... ; WHILE (iterate) { alpha, U, G, Y, X, R, check; IF (continue) { F, W,
//         gamma, P, V } }
// The check kernels count k, record the residual, decide (converged, diverged, stalled, maxit,
// breakdown) and set the conditions.  The host launches the graph once and synchronises once for
// all jobs; every wait is a graph dependency, none is a spin.
namespace {

constexpr int GRAPH_STALLED = 100;   // run status: the low-precision preconditioner stopped improving

struct GraphCtl {
  int k, maxit_run, stall, k_best, status, L, hist_len, hist_n;
  int mode, may_fall_back, restore, iters, restarts, max_restarts, fallbacks, stall_window, maxit;
  int runs[2], iters_mode[2];
  double tol, div, best;
  double bnorm2[WD_LMAX];
  double rec[WD_LMAX];
  double true2[WD_LMAX];
};

__device__ double graph_max_rel(const double* n2, GraphCtl* g) {
  double m = 0.0;
  for (int i = 0; i < g->L; ++i) {
    const double r = sqrt(n2[i]) / sqrt(g->bnorm2[i]);
    g->rec[i] = r;
    if (!(r <= m)) m = r;
  }
  return m;
}

__device__ void graph_record(GraphCtl* g, double* hist, double m) {
  if (hist && g->hist_n < g->hist_len) hist[g->hist_n] = m;
  if (g->hist_n < g->hist_len) g->hist_n += 1;
}

// Start of a pass: open the branch of the current mode.
__global__ void graph_phase_begin(const GraphCtl* g, cudaGraphConditionalHandle hrun0,
                                  cudaGraphConditionalHandle hrun1, int two_modes) {
  if (threadIdx.x != 0) return;
  cudaGraphSetConditional(hrun0, g->mode == 0 ? 1u : 0u);
  if (two_modes) cudaGraphSetConditional(hrun1, g->mode == 1 ? 1u : 0u);
}

// X = X_0 when the pass is the first one after a fallback.
__global__ void graph_restore_x(const GraphCtl* g, double2* X, const double2* X0, long long n) {
  if (!g->restore) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    X[i] = X0[i];
}

// After R_0 of a run: the first residual check (k = 0).
__global__ void graph_init_check(const SolverState* st, GraphCtl* g, double* hist,
                                 cudaGraphConditionalHandle hloop) {
  if (threadIdx.x != 0) return;
  const double m = graph_max_rel(st->rnorm2, g);
  g->restore = 0;
  g->k = 0;
  g->best = m;
  g->k_best = 0;
  g->maxit_run = g->maxit - g->iters;
  g->stall = g->mode == 0 && g->may_fall_back ? g->stall_window : 0;
  graph_record(g, hist, m);
  int done = 0, status = WD_OK;
  if (!isfinite(m)) { done = 1; status = WD_BREAKDOWN; }
  else if (m <= g->tol) { done = 1; status = WD_OK; }
  else if (g->maxit_run <= 0) { done = 1; status = WD_NOT_CONVERGED; }
  g->status = status;
  cudaGraphSetConditional(hloop, done ? 0u : 1u);
}

__global__ void graph_iter_check(const SolverState* st, GraphCtl* g, double* hist,
                                 cudaGraphConditionalHandle hloop, cudaGraphConditionalHandle htail) {
  if (threadIdx.x != 0) return;
  int done = 0, status = WD_OK;
  if (st->status != ST_OK) {
    done = 1;
    status = WD_BREAKDOWN;                    // the update was skipped: k stays
  } else {
    g->k += 1;
    const double m = graph_max_rel(st->rnorm2, g);
    graph_record(g, hist, m);
    if (!isfinite(m)) { done = 1; status = WD_BREAKDOWN; }
    else if (m <= g->tol) { done = 1; status = WD_OK; }
    else if (m > g->div) { done = 1; status = WD_DIVERGED; }
    else {
      if (m < g->best) { g->best = m; g->k_best = g->k; }
      if (g->stall > 0 && g->k - g->k_best >= g->stall) { done = 1; status = GRAPH_STALLED; }
      else if (g->k >= g->maxit_run) { done = 1; status = WD_NOT_CONVERGED; }
    }
  }
  g->status = status;
  cudaGraphSetConditional(hloop, done ? 0u : 1u);
  cudaGraphSetConditional(htail, done ? 0u : 1u);
}

// End of a pass, after the true residual ||b_i - A x_i||^2 is in true2: fall back to the FP64
// preconditioner from X_0 (a stalled, broken-down or diverged low-precision run), restart from X
// (converged recursively but not truly), or stop -- the decisions of bbicggr_solve.
__global__ void graph_phase_end(GraphCtl* g, cudaGraphConditionalHandle hphase) {
  if (threadIdx.x != 0) return;
  g->iters += g->k;
  g->runs[g->mode] += 1;
  g->iters_mode[g->mode] += g->k;
  int status = g->status, again = 0;
  if (g->mode == 0 && g->may_fall_back && g->iters < g->maxit &&
      (status == GRAPH_STALLED || status == WD_BREAKDOWN || status == WD_DIVERGED)) {
    g->mode = 1;
    g->restore = 1;
    g->fallbacks += 1;
    again = 1;
  } else {
    if (status == GRAPH_STALLED) status = WD_NOT_CONVERGED;
    double mtrue = 0.0;
    for (int i = 0; i < g->L; ++i) {
      const double r = sqrt(g->true2[i]) / sqrt(g->bnorm2[i]);
      if (!(r <= mtrue)) mtrue = r;
    }
    if (status == WD_OK && !(mtrue <= g->tol)) {
      if (g->restarts >= g->max_restarts || g->iters >= g->maxit) status = WD_NOT_CONVERGED;
      else { g->restarts += 1; again = 1; }
    }
    g->status = status;
  }
  cudaGraphSetConditional(hphase, again ? 1u : 0u);
}

// Enqueue `fn` on the context's capture stream as nodes of graph `g` after `deps`; the leaf nodes
// of what was captured are returned in *leaves.
template <class Fn>
int capture_into(wd_ctx* c, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, Fn fn,
                 std::vector<cudaGraphNode_t>* leaves) {
  cudaStream_t s = c->capture_stream;
  CU(cudaStreamBeginCaptureToGraph(s, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                   deps.size(), cudaStreamCaptureModeThreadLocal));
  int rc = fn(s);
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* d = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &d, nullptr, &nd);
  if (e == cudaSuccess && leaves) leaves->assign(d, d + nd);
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(s, &out);
  if (rc != WD_OK) return rc;
  CU(e);
  CU(e2);
  return WD_OK;
}

// M applied so that the result always lands in `out` (fixed buffers for a graph body).
int precondition_into(wd_ctx* c, const double* R, double* out, double* tmp, int L, int j,
                      int precision, cudaStream_t s) {
  const bool to_tmp_first = precision == 0 && j > 0 && j % 2 == 0;
  double* res = nullptr;
  CHECK(precondition(c, R, to_tmp_first ? tmp : out, to_tmp_first ? out : tmp, &res, L, j,
                     precision, nullptr, s));
  if (res != out) { set_err("internal: preconditioner result buffer"); return WD_ECUDA; }
  return WD_OK;
}

struct JobPtrs {
  const double* B;
  double* X;
  double* X0;             // X_0, kept for a fallback (null when the job cannot fall back)
  int L, j, mode;
  bool df;
  double tol;
};

// One run of block BiCGGR from the current X with preconditioner `mode` into graph `RB`.
int build_run(wd_ctx* c, const JobPtrs& jp, int mode, bool df, bool restore, cudaGraph_t RB) {
  const Op& op = c->op;
  const int L = jp.L, j = jp.j;
  const long long rows = (long long)op.g.V * 12;
  const size_t bytes = block_bytes(c, L);
  double* R = c->blk[B_R].d();
  double* P = c->blk[B_P].d();
  double* V = c->blk[B_V].d();
  double* W = c->blk[B_W].d();
  double* U = c->blk[B_U].d();
  double* Y = c->blk[B_Y].d();
  double* Rt = c->blk[B_RT].d();
  double* F = c->blk[B_F].d();
  double* Gk = c->blk[B_G].d();
  double* T = c->blk[B_T].d();
  double2* part = static_cast<double2*>(c->part.p);
  SolverState* st = c->st;
  GraphCtl* g = static_cast<GraphCtl*>(c->gctl);
  double* hist = c->ghist;

  cudaGraphConditionalHandle hloop;
  CU(cudaGraphConditionalHandleCreate(&hloop, RB, 0, 0));
  std::vector<cudaGraphNode_t> pre_leaves, a_leaves, dummy;
  // R_0, P_0, R~_0, R~_0^H R_0, the first check, F_0, V_0 = W_0, traces, R~_0^H V_0
  CHECK(capture_into(c, RB, {}, [&](cudaStream_t s) -> int {
    if (restore) {
      graph_restore_x<<<1024, 256, 0, s>>>(g, reinterpret_cast<double2*>(jp.X),
                                           reinterpret_cast<const double2*>(jp.X0), rows * L);
      CU(cudaGetLastError());
    }
    CU(cudaMemsetAsync(&st->status, 0, sizeof(int), s));
    LAUNCH(WD_K_RESID, stencil_kernels(op), launch_resid_f64(op, jp.X, jp.B, R, L, s));
    LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(P, R, bytes, cudaMemcpyDeviceToDevice, s));
    LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(Rt, R, bytes, cudaMemcpyDeviceToDevice, s));
    LAUNCH(WD_K_GRAM, 2, launch_gram(Rt, R, L, rows, part, st, GRAM_RTR, true, s));
    graph_init_check<<<1, 32, 0, s>>>(st, g, hist, hloop);
    CU(cudaGetLastError());
    CHECK(precondition_into(c, R, F, T, L, j, mode, s));
    LAUNCH(WD_K_APPLY, stencil_kernels(op), launch_apply_f64(op, F, W, L, s));
    LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(V, W, bytes, cudaMemcpyDeviceToDevice, s));
    LAUNCH(WD_K_TRACE, 2, launch_traces(W, R, L, rows, part, st, s));
    LAUNCH(WD_K_GRAM, 2, launch_gram(Rt, V, L, rows, part, st, GRAM_RTV, false, s));
    return WD_OK;
  }, &pre_leaves));
  // the outer iteration
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hloop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t nwhile;
  CU(cudaGraphAddNode(&nwhile, RB, pre_leaves.data(), nullptr, pre_leaves.size(), &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  cudaGraphConditionalHandle htail;
  CU(cudaGraphConditionalHandleCreate(&htail, body, 0, 0));
  CHECK(capture_into(c, body, {}, [&](cudaStream_t s) -> int {
    LAUNCH(WD_K_SOLVE_LL, 1, launch_solve_alpha(st, L, s));
    LAUNCH(WD_K_UPDATE_U, 1, launch_update_u(P, V, U, L, rows, st, s, df));
    CHECK(precondition_into(c, U, Gk, T, L, j, mode, s));
    LAUNCH(WD_K_APPLY, stencil_kernels(op), launch_apply_f64(op, Gk, Y, L, s));
    LAUNCH(WD_K_UPDATE_XR, 2, launch_update_xr(jp.X, F, Gk, R, W, Y, Rt, L, rows, part, st, s, df));
    graph_iter_check<<<1, 32, 0, s>>>(st, g, hist, hloop, htail);
    CU(cudaGetLastError());
    return WD_OK;
  }, &a_leaves));
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = htail;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t nif;
  CU(cudaGraphAddNode(&nif, body, a_leaves.data(), nullptr, a_leaves.size(), &ip));
  cudaGraph_t tail = ip.conditional.phGraph_out[0];
  CHECK(capture_into(c, tail, {}, [&](cudaStream_t s) -> int {
    CHECK(precondition_into(c, R, F, T, L, j, mode, s));
    LAUNCH(WD_K_APPLY, stencil_kernels(op), launch_apply_f64(op, F, W, L, s));
    LAUNCH(WD_K_TRACE, 2, launch_traces(W, R, L, rows, part, st, s));
    LAUNCH(WD_K_SOLVE_LL, 1, launch_solve_gamma(st, L, s));
    LAUNCH(WD_K_UPDATE_PV, 2, launch_update_pv(P, V, R, W, U, Y, Rt, L, rows, part, st, s, df));
    return WD_OK;
  }, &dummy));
  return WD_OK;
}

// Adds a conditional node of `type` (handle h) to `graph` after `deps`; its body is returned.
int add_conditional(cudaGraph_t graph, const std::vector<cudaGraphNode_t>& deps,
                    cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    cudaGraphNode_t* node, cudaGraph_t* body) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  CU(cudaGraphAddNode(node, graph, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p));
  *body = p.conditional.phGraph_out[0];
  return WD_OK;
}

int build_job(wd_ctx* c, const JobPtrs& jp, cudaGraph_t G) {
  const Op& op = c->op;
  const int L = jp.L;
  const long long rows = (long long)op.g.V * 12;
  const size_t bytes = block_bytes(c, L);
  double* T = c->blk[B_T].d();
  double2* part = static_cast<double2*>(c->part.p);
  GraphCtl* g = static_cast<GraphCtl*>(c->gctl);
  const bool two_modes = jp.X0 != nullptr;

  cudaGraphConditionalHandle hphase;
  CU(cudaGraphConditionalHandleCreate(&hphase, G, 1, cudaGraphCondAssignDefault));
  std::vector<cudaGraphNode_t> pre_leaves, begin_leaves, dummy;
  CHECK(capture_into(c, G, {}, [&](cudaStream_t s) -> int {
    LAUNCH(WD_K_COLNORM, 2, launch_colnorms(jp.B, L, rows, part, g->bnorm2, s));
    if (two_modes)
      LAUNCH(WD_K_COPY, 0, cudaMemcpyAsync(jp.X0, jp.X, bytes, cudaMemcpyDeviceToDevice, s));
    return WD_OK;
  }, &pre_leaves));
  cudaGraphNode_t nphase, nrun0, nrun1 = nullptr;
  cudaGraph_t pass, rb0, rb1 = nullptr;
  CHECK(add_conditional(G, pre_leaves, hphase, cudaGraphCondTypeWhile, &nphase, &pass));
  cudaGraphConditionalHandle hrun0, hrun1 = 0;
  CU(cudaGraphConditionalHandleCreate(&hrun0, pass, 0, 0));
  if (two_modes) CU(cudaGraphConditionalHandleCreate(&hrun1, pass, 0, 0));
  CHECK(capture_into(c, pass, {}, [&](cudaStream_t s) -> int {
    graph_phase_begin<<<1, 32, 0, s>>>(g, hrun0, hrun1, two_modes ? 1 : 0);
    CU(cudaGetLastError());
    return WD_OK;
  }, &begin_leaves));
  CHECK(add_conditional(pass, begin_leaves, hrun0, cudaGraphCondTypeIf, &nrun0, &rb0));
  CHECK(build_run(c, jp, jp.mode, jp.df, false, rb0));
  if (two_modes) {
    CHECK(add_conditional(pass, {nrun0}, hrun1, cudaGraphCondTypeIf, &nrun1, &rb1));
    CHECK(build_run(c, jp, PM_F64, false, true, rb1));
  }
  // the true residual of the pass, then the decision
  CHECK(capture_into(c, pass, {two_modes ? nrun1 : nrun0}, [&](cudaStream_t s) -> int {
    LAUNCH(WD_K_RESID, stencil_kernels(op), launch_resid_f64(op, jp.X, jp.B, T, L, s));
    LAUNCH(WD_K_COLNORM, 2, launch_colnorms(T, L, rows, part, g->true2, s));
    graph_phase_end<<<1, 32, 0, s>>>(g, hphase);
    CU(cudaGetLastError());
    return WD_OK;
  }, &dummy));
  return WD_OK;
}

}  // namespace

extern "C" int bbicggr_solve_batch(bbicggr_job* jobs, int njobs, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!jobs || njobs < 1) { set_err("no jobs"); return WD_EINVAL; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < njobs; ++i) {
    bbicggr_job& jb = jobs[i];
    wd_ctx* c = jb.ctx;
    if (!c) { set_err("job %d: ctx is NULL", i); return WD_EINVAL; }
    if (c->dom_on) { set_err("job %d: a domain-decomposed context cannot join a batch", i); return WD_EINVAL; }
    for (int k = 0; k < i; ++k)
      if (jobs[k].ctx == c) { set_err("jobs %d and %d share a context", k, i); return WD_EINVAL; }
    CHECK(check_L(jb.L));
    if (jb.j < 0 || !(jb.tol > 0.0)) { set_err("job %d: j < 0 or tol <= 0", i); return WD_EINVAL; }
    if (!jb.B || !jb.X || !is_device_ptr(jb.B) || !is_device_ptr(jb.X)) {
      set_err("job %d: B and X must be device buffers", i);
      return WD_EINVAL;
    }
    const bbicggr_opts& o = jb.opts;
    if (o.maxit < 0 || !(o.div_thresh > 0.0) || o.stall_window < 0 ||
        o.precision < 0 || o.precision > 5) {
      set_err("job %d: invalid options", i);
      return WD_EINVAL;
    }
  }
  // workspace, tuning, network buffers and control blocks before any capture
  for (int i = 0; i < njobs; ++i) {
    bbicggr_job& jb = jobs[i];
    wd_ctx* c = jb.ctx;
    CHECK(ensure_workspace(c, jb.L));
    const int mode = precond_mode(jb.opts);
    if ((mode == PM_F32 || mode == PM_BF16) && jb.j >= 2)
      CHECK(ensure_workspace_lp(c, lp_storage(mode), jb.L, s));
    if (mode == PM_DF && jb.j >= 2) CHECK(ensure_workspace_df(c, jb.L, s));
    if (mode == PM_NET) CHECK(wd_net_prepare(c, jb.opts.net, jb.L));
    if (!c->gctl) CU(cudaMalloc(&c->gctl, sizeof(GraphCtl)));
    const int hl = jb.opts.history ? jb.opts.history_len : 0;
    if (hl > c->ghist_len) {
      cudaFree(c->ghist);
      c->ghist = nullptr;
      c->ghist_len = 0;
      CU(cudaMalloc(&c->ghist, hl * sizeof(double)));
      c->ghist_len = hl;
    }
    if (!c->capture_stream) CU(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    const bool may_fall_back = mode != PM_F64 && jb.opts.stall_window > 0;
    if (may_fall_back) CHECK(c->blk[B_X0].ensure(block_bytes(c, jb.L)));
    GraphCtl h = {};
    h.maxit = jb.opts.maxit;
    h.stall_window = jb.opts.stall_window;
    h.may_fall_back = may_fall_back ? 1 : 0;
    h.max_restarts = jb.opts.max_restarts;
    h.L = jb.L;
    h.hist_len = hl;
    h.tol = jb.tol;
    h.div = jb.opts.div_thresh;
    CU(cudaMemcpyAsync(c->gctl, &h, sizeof(GraphCtl), cudaMemcpyHostToDevice, s));
  }
  CU(cudaStreamSynchronize(s));
  cudaGraph_t G = nullptr;
  CU(cudaGraphCreate(&G, 0));
  int rc = WD_OK;
  for (int i = 0; i < njobs && rc == WD_OK; ++i) {
    bbicggr_job& jb = jobs[i];
    wd_ctx* c = jb.ctx;
    const bool timing = c->prof.timing;
    c->prof.timing = false;                 // no event nodes in the graph
    c->active_net = jb.opts.net;
    c->net_bf16 = jb.opts.net && jb.opts.precision == 3;
    const int mode = precond_mode(jb.opts);
    double* X0 = mode != PM_F64 && jb.opts.stall_window > 0 ? c->blk[B_X0].d() : nullptr;
    JobPtrs jp{static_cast<const double*>(jb.B), static_cast<double*>(jb.X), X0, jb.L, jb.j,
               mode, jb.opts.precision == 2 || jb.opts.precision == 5, jb.tol};
    rc = build_job(c, jp, G);
    c->prof.timing = timing;
  }
  cudaGraphExec_t exec = nullptr;
  if (rc == WD_OK) {
    cudaError_t e = cudaGraphInstantiate(&exec, G, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_err("graph solve failed: %s", cudaGetErrorString(e));
      rc = WD_ECUDA;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  cudaGraphDestroy(G);
  if (rc != WD_OK) return rc;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = WD_OK;
  for (int i = 0; i < njobs; ++i) {
    bbicggr_job& jb = jobs[i];
    wd_ctx* c = jb.ctx;
    GraphCtl h;
    CU(cudaMemcpy(&h, c->gctl, sizeof(GraphCtl), cudaMemcpyDeviceToHost));
    bbicggr_info& in = jb.info;
    const int jeff = jb.opts.net ? 0 : jb.j;    // run 0: the job's preconditioner; run 1: FP64 Jacobi
    double mtrue = 0.0, mrec = 0.0;
    double tr[WD_LMAX];
    for (int k = 0; k < jb.L; ++k) {
      tr[k] = std::sqrt(h.true2[k]) / std::sqrt(h.bnorm2[k]);
      if (!(tr[k] <= mtrue)) mtrue = tr[k];
      if (!(h.rec[k] <= mrec)) mrec = h.rec[k];
    }
    int status = h.status;
    if (status == WD_OK && !(mtrue <= jb.tol)) status = WD_NOT_CONVERGED;
    in.status = status;
    in.iters = h.iters;
    in.restarts = h.restarts;
    in.fallbacks = h.fallbacks;
    in.mvm_paper = (long long)jb.L * (2LL * (jeff + 1) * h.iters_mode[0] + h.runs[0] +
                                      2LL * (jb.j + 1) * h.iters_mode[1] + h.runs[1]);
    in.mvm_actual = -1;
    in.max_rec_resid = mrec;
    in.max_true_resid = mtrue;
    if (in.rec_resid) std::memcpy(in.rec_resid, h.rec, jb.L * sizeof(double));
    if (in.true_resid) std::memcpy(in.true_resid, tr, jb.L * sizeof(double));
    in.history_count = 0;
    if (jb.opts.history && h.hist_n > 0) {
      const int n = std::min(h.hist_n, h.hist_len);
      CU(cudaMemcpy(jb.opts.history, c->ghist, n * sizeof(double), cudaMemcpyDeviceToHost));
      in.history_count = n;
    }
    in.seconds = secs;
    c->solved_L = jb.L;
    if (status != WD_OK && worst == WD_OK) worst = status;
  }
  return worst;
}

extern "C" int wd_copy_residual(wd_ctx* c, void* R, int L, void* stream) {
  if (!c || !R) { set_err("ctx or R is NULL"); return WD_EINVAL; }
  if (c->solved_L == 0 || L != c->solved_L) {
    set_err("no solve with L = %d on this context (last: %d)", L, c->solved_L);
    return WD_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CU(cudaMemcpyAsync(R, c->blk[B_R].d(), block_bytes(c, L), cudaMemcpyDefault, s));
  CU(cudaStreamSynchronize(s));
  return WD_OK;
}
