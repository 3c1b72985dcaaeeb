// jacobi_precond_noalloc: the Jacobi preconditioner G = M R without any allocation.
//
// Some callers cannot let a library call cudaMalloc: a framework whose caching allocator already
// owns the free device memory (an outside cudaMalloc can fail or fragment it), or a latency-bound
// loop that cannot afford cudaMalloc/cudaFree and the device synchronisation cudaFree implies.
// jacobi_precond itself takes its ping-pong block from the context's solver workspace, which it
// allocates on first use.  This variant instead takes that block from the file-scope array below.
// wd_create loads the array on its device (noalloc_reserve), so every GPU on which a context has
// been created holds the 32 MiB from then until the process exits.
#include <cstdint>

#include "../../include/bbicggr.h"
#include "internal.h"

namespace {

// Scratch for the ping-pong block of the Jacobi sweeps: at most NOALLOC_SCRATCH_DOUBLES reals,
// i.e. 12 * V * L complex numbers <= NOALLOC_SCRATCH_DOUBLES / 2 (32 MiB).
constexpr size_t NOALLOC_SCRATCH_DOUBLES = size_t(4) << 20;
constexpr long long NOALLOC_MAX_ELEMENTS = (long long)(NOALLOC_SCRATCH_DOUBLES / 2);
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

// Device address of the scratch array on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, so the address comes from cudaGetSymbolAddress
// with that device current.  It is looked up on every call rather than cached: once the module is
// loaded the lookup allocates nothing and is cheap, and a cached address would go stale if the
// device's primary context were reset and the module reloaded elsewhere.
int scratch_for_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    wd_set_error("jacobi_precond_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? WD_ENOMEM : WD_ECUDA;
  }
  *out = static_cast<double*>(p);
  return WD_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// With CUDA's lazy module loading, the module that holds g_noalloc_scratch -- and with it the
// 32 MiB -- is loaded the first time something on the device refers to it.  wd_create calls this
// on the context's device so that the array is taken at a predictable point, before a caller's
// caching allocator may have claimed the free memory, and never inside a later call.
int noalloc_reserve(void) {
  double* p = nullptr;
  return scratch_for_current_device(&p);
}

extern "C" int jacobi_precond_noalloc(wd_ctx* ctx, const void* R, void* G, int L, int j,
                                      void* stream) {
  if (!ctx) { wd_set_error("ctx is NULL"); return WD_EINVAL; }
  if (L < 1 || L > WD_LMAX) { wd_set_error("L = %d outside [1, %d]", L, WD_LMAX); return WD_EINVAL; }
  if (j < 0) { wd_set_error("j = %d < 0", j); return WD_EINVAL; }
  if (!R || !G) { wd_set_error("R or G is NULL"); return WD_EINVAL; }
  if (!on_device(R) || !on_device(G)) {
    wd_set_error("jacobi_precond_noalloc takes device buffers only (host buffers need staging)");
    return WD_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(R) % 16 || reinterpret_cast<uintptr_t>(G) % 16) {
    wd_set_error("R and G must be 16-byte aligned");
    return WD_EINVAL;
  }
  const Op& op = *wd_ctx_op(ctx);
  const long long elems = (long long)op.g.V * 12 * L;   // complex numbers in one block
  if (elems > NOALLOC_MAX_ELEMENTS) {
    wd_set_error("jacobi_precond_noalloc: 12*V*L = %lld complex numbers exceeds the static "
                 "scratch of %lld (32 MiB); use jacobi_precond", elems, NOALLOC_MAX_ELEMENTS);
    return WD_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != wd_ctx_device(ctx)) {
    cudaGetLastError();
    wd_set_error("jacobi_precond_noalloc: the current device (%d) is not the context's device (%d)",
                 dev, wd_ctx_device(ctx));
    return WD_EINVAL;
  }
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != WD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double* r = static_cast<const double*>(R);
  double* g = static_cast<double*>(G);
  cudaError_t e = cudaSuccess;
  if (j == 0) {
    e = cudaMemcpyAsync(g, r, (size_t)elems * 16, cudaMemcpyDeviceToDevice, s);
    wd_ctx_count_launches(ctx, WD_K_COPY, 0);
  } else {
    // j sweeps alternate between two blocks; start in G when j is odd so the last lands in G.
    double* cur = (j % 2 == 1) ? g : scratch;
    double* nxt = (j % 2 == 1) ? scratch : g;
    e = launch_site_inverse_f64(op, r, cur, L, s);
    wd_ctx_count_launches(ctx, WD_K_SITE_INV, 1);
    for (int i = 1; i < j && e == cudaSuccess; ++i) {
      e = launch_jacobi_f64(op, cur, r, nxt, L, s);
      wd_ctx_count_launches(ctx, WD_K_JACOBI, stencil_kernels(op));
      double* t = cur;
      cur = nxt;
      nxt = t;
    }
  }
  if (e != cudaSuccess) {
    wd_set_error("jacobi_precond_noalloc: %s", cudaGetErrorString(e));
    return WD_ECUDA;
  }
  return WD_OK;
}
