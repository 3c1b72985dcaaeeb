// C-ABI of the learned preconditioner network (declared in include/bbicggr.h): weights, Adam
// state and the activation workspaces of one network (one per context it runs on), inference
// G = N(R), and one training step on pairs (R, E = A^{-1} R).  The kernels live in net.cu; see its
// header for the network.
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bbicggr.h"
#include "internal.h"

namespace {

bool dev_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define NCU(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      wd_set_error("%s failed: %s", #call, cudaGetErrorString(e_));                 \
      return e_ == cudaErrorMemoryAllocation ? WD_ENOMEM : WD_ECUDA;                \
    }                                                                               \
  } while (0)
#define NCHECK(rc)               \
  do {                           \
    int rc_ = (rc);              \
    if (rc_ != WD_OK) return rc_; \
  } while (0)

constexpr int NET_MAX_LAYERS = 16;
constexpr int NET_BLOCKS = 608;     // reduction blocks of the loss and weight-gradient kernels

}  // namespace

// Activations (and, for training, the loss and gradient reductions) for one lattice volume V and
// L.  A network keeps one workspace per context it is applied on, so that solves on different
// contexts -- the jobs of one batch graph run at the same time -- never share buffers, and one
// for training (key nullptr), whose calls run one after another.
struct NetWs {
  const void* key = nullptr;
  bool train = false;
  long long V = 0;
  int L = 0;
  std::vector<float*> act;      // act[l]: input of layer l; act[layers]: output
  float* dA = nullptr;
  float* dB = nullptr;
  double* wcol = nullptr;
  double* loss = nullptr;
  double* lpart = nullptr;
  double2* wpart = nullptr;
  double* norms = nullptr;
  void release() {
    for (float* a : act) cudaFree(a);
    act.clear();
    cudaFree(dA); cudaFree(dB); cudaFree(wcol); cudaFree(loss); cudaFree(lpart); cudaFree(wpart);
    cudaFree(norms);
    dA = dB = nullptr; wcol = loss = lpart = norms = nullptr; wpart = nullptr;
    V = 0; L = 0;
  }
};

struct wd_net {
  int layers = 0, hidden = 0;
  std::vector<int> ch;          // channels: ch[0] = 1, ch[layers] = 1
  std::vector<size_t> off;      // complex offset of each layer's weights
  size_t nw = 0;                // complex weights in total
  float2* W = nullptr;
  float2* Wadj = nullptr;       // scratch for one layer's adjoint weights
  double2* G = nullptr;         // d loss / d conj(W) of the last loss_grad call
  float2* m = nullptr;
  float2* v = nullptr;
  int t = 0;                    // Adam steps taken
  std::vector<NetWs*> ws;
  void free_ws() {
    for (NetWs* w : ws) { w->release(); delete w; }
    ws.clear();
  }
};

namespace {

size_t chan_floats(long long V, int L) { return (size_t)12 * V * L * 2; }

// The workspace of (key, train) sized for (V, L), allocated or resized here unless `s` is being
// captured into a graph, where allocation is not allowed (wd_net_prepare runs before a capture).
int net_workspace(wd_net* n, const void* key, bool train, long long V, int L, cudaStream_t s,
                  NetWs** out) {
  NetWs* w = nullptr;
  for (NetWs* e : n->ws)
    if (e->key == key && e->train == train) w = e;
  if (w && w->V == V && w->L == L) { *out = w; return WD_OK; }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NCU(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    wd_set_error("network workspace not prepared for V = %lld, L = %d before the capture", V, L);
    return WD_EINVAL;
  }
  if (!w) {
    w = new (std::nothrow) NetWs();
    if (!w) { wd_set_error("host allocation failed"); return WD_ENOMEM; }
    w->key = key;
    w->train = train;
    n->ws.push_back(w);
  }
  w->release();
  const size_t cf = chan_floats(V, L) * sizeof(float);
  w->act.assign(n->layers + 1, nullptr);
  for (int l = 0; l <= n->layers; ++l) NCU(cudaMalloc(&w->act[l], cf * n->ch[l]));
  if (train) {
    int maxc = 1;
    for (int c : n->ch) maxc = c > maxc ? c : maxc;
    NCU(cudaMalloc(&w->dA, cf * maxc));
    NCU(cudaMalloc(&w->dB, cf * maxc));
    NCU(cudaMalloc(&w->wcol, WD_LMAX * sizeof(double)));
    NCU(cudaMalloc(&w->loss, sizeof(double)));
    NCU(cudaMalloc(&w->lpart, NET_BLOCKS * sizeof(double)));
    NCU(cudaMalloc(&w->norms, (size_t)(PART_STRIDE * NET_BLOCKS + WD_LMAX) * sizeof(double2)));
    size_t maxne = 0;
    for (int l = 0; l < n->layers; ++l) {
      const size_t ne = (size_t)9 * n->ch[l + 1] * n->ch[l] * 16;
      maxne = ne > maxne ? ne : maxne;
    }
    NCU(cudaMalloc(&w->wpart, (size_t)NET_BLOCKS * maxne * sizeof(double2)));
  }
  w->V = V;
  w->L = L;
  *out = w;
  return WD_OK;
}

// act[layers] = N(act[0]) (activations of every layer kept); bf16: the activations are stored
// in BF16 (the buffers, sized for FP32, hold them in their first half).
int net_forward(const Op& op, wd_net* n, NetWs* w, int L, cudaStream_t s, bool bf16 = false) {
  for (int l = 0; l < n->layers; ++l) {
    if (bf16)
      NCU(net_launch_layer_bf16(op, w->act[l], w->act[l + 1], n->W + n->off[l], n->ch[l],
                                n->ch[l + 1], L, s));
    else
      NCU(net_launch_layer(op, w->act[l], w->act[l + 1], n->W + n->off[l], n->ch[l],
                           n->ch[l + 1], L, s));
  }
  return WD_OK;
}

__global__ void weights_from_c128(const double* in, float2* out, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)in[2 * i], (float)in[2 * i + 1]);
}
__global__ void weights_to_c128(const float2* in, double* out, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) { out[2 * i] = in[i].x; out[2 * i + 1] = in[i].y; }
}
__global__ void wcol_kernel(const double* norm2, double* wcol, int L) {
  const int i = threadIdx.x;
  if (i < L) wcol[i] = 1.0 / ((double)L * norm2[i]);
}

int set_weights(wd_net* n, const void* w) {
  double* tmp = nullptr;
  const double* src = static_cast<const double*>(w);
  if (!dev_ptr(w)) {
    NCU(cudaMalloc(&tmp, n->nw * 16));
    NCU(cudaMemcpy(tmp, w, n->nw * 16, cudaMemcpyHostToDevice));
    src = tmp;
  }
  weights_from_c128<<<(unsigned)((n->nw + 255) / 256), 256>>>(src, n->W, n->nw);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(tmp);
  NCU(e);
  NCU(cudaMemset(n->m, 0, n->nw * sizeof(float2)));
  NCU(cudaMemset(n->v, 0, n->nw * sizeof(float2)));
  n->t = 0;
  return WD_OK;
}

}  // namespace

// Internal: allocate the network's workspace for this context and L (before a stream capture).
int wd_net_prepare(wd_ctx* ctx, wd_net* n, int L) {
  NetWs* w;
  return net_workspace(n, ctx, false, wd_ctx_op(ctx)->g.V, L, nullptr, &w);
}

// Internal: G = N(R) for device blocks R, G (site-major FP64), used by the solver.
int wd_net_precondition(wd_ctx* ctx, wd_net* n, const double* R, double* G, int L, bool bf16,
                        cudaStream_t s) {
  const Op& op = *wd_ctx_op(ctx);
  NetWs* w;
  NCHECK(net_workspace(n, ctx, false, op.g.V, L, s, &w));
  NCU(net_launch_to_cm(R, w->act[0], op.g.V, L, bf16, s));
  NCHECK(net_forward(op, n, w, L, s, bf16));
  NCU(net_launch_from_cm(w->act[n->layers], G, op.g.V, L, bf16, s));
  return WD_OK;
}

extern "C" {

int wd_net_create(wd_net** out, int layers, int hidden, const void* weights) {
  if (!out) { wd_set_error("out is NULL"); return WD_EINVAL; }
  *out = nullptr;
  if (layers < 1 || layers > NET_MAX_LAYERS || (hidden != 1 && hidden != 2 && hidden != 4) ||
      (layers == 1 && hidden != 1)) {
    wd_set_error("network of %d layers x %d hidden channels not available (hidden 1, 2 or 4)",
                 layers, hidden);
    return WD_EINVAL;
  }
  if (!weights) { wd_set_error("weights is NULL"); return WD_EINVAL; }
  wd_net* n = new (std::nothrow) wd_net();
  if (!n) { wd_set_error("host allocation failed"); return WD_ENOMEM; }
  n->layers = layers;
  n->hidden = hidden;
  n->ch.assign(layers + 1, hidden);
  n->ch[0] = 1;
  n->ch[layers] = 1;
  for (int l = 0; l < layers; ++l) {
    n->off.push_back(n->nw);
    n->nw += (size_t)9 * n->ch[l + 1] * n->ch[l] * 16;
  }
  int rc = WD_OK;
  if (cudaMalloc(&n->W, n->nw * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&n->Wadj, n->nw * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&n->G, n->nw * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&n->m, n->nw * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&n->v, n->nw * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    wd_set_error("device allocation for the network failed");
    rc = WD_ENOMEM;
  }
  if (rc == WD_OK) rc = set_weights(n, weights);
  if (rc != WD_OK) { wd_net_destroy(n); return rc; }
  *out = n;
  return WD_OK;
}

void wd_net_destroy(wd_net* n) {
  if (!n) return;
  n->free_ws();
  cudaFree(n->W); cudaFree(n->Wadj); cudaFree(n->G); cudaFree(n->m); cudaFree(n->v);
  delete n;
}

long long wd_net_num_weights(const wd_net* n) { return n ? (long long)n->nw : -1; }

int wd_net_set_weights(wd_net* n, const void* weights) {
  if (!n || !weights) { wd_set_error("net or weights is NULL"); return WD_EINVAL; }
  return set_weights(n, weights);
}

int wd_net_get_weights(const wd_net* n, void* out) {
  if (!n || !out) { wd_set_error("net or out is NULL"); return WD_EINVAL; }
  double* tmp = nullptr;
  NCU(cudaMalloc(&tmp, n->nw * 16));
  weights_to_c128<<<(unsigned)((n->nw + 255) / 256), 256>>>(n->W, tmp, n->nw);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(out, tmp, n->nw * 16, cudaMemcpyDefault);
  cudaFree(tmp);
  NCU(e);
  return WD_OK;
}

int wd_net_apply(wd_ctx* ctx, wd_net* n, const void* R, void* G, int L, int bf16, void* stream) {
  if (!ctx || !n || !R || !G) { wd_set_error("NULL argument"); return WD_EINVAL; }
  if (bf16 != 0 && bf16 != 1) { wd_set_error("bf16 = %d not in {0, 1}", bf16); return WD_EINVAL; }
  if (L < 1 || L > WD_LMAX) { wd_set_error("L = %d outside [1, %d]", L, WD_LMAX); return WD_EINVAL; }
  if (!dev_ptr(R) || !dev_ptr(G)) { wd_set_error("wd_net_apply takes device buffers"); return WD_EINVAL; }
  return wd_net_precondition(ctx, n, static_cast<const double*>(R), static_cast<double*>(G), L,
                             bf16 != 0, static_cast<cudaStream_t>(stream));
}

int wd_net_loss_grad(wd_ctx* ctx, wd_net* n, const void* R, const void* E, int L, double* loss,
                     void* grad, void* stream) {
  if (!ctx || !n || !R || !E) { wd_set_error("NULL argument"); return WD_EINVAL; }
  if (L < 1 || L > WD_LMAX) { wd_set_error("L = %d outside [1, %d]", L, WD_LMAX); return WD_EINVAL; }
  if (!dev_ptr(R) || !dev_ptr(E)) { wd_set_error("wd_net_loss_grad takes device buffers"); return WD_EINVAL; }
  const Op& op = *wd_ctx_op(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long V = op.g.V;
  NetWs* w;
  NCHECK(net_workspace(n, nullptr, true, V, L, s, &w));
  // forward, keeping the activations
  NCU(net_launch_to_cm(static_cast<const double*>(R), w->act[0], (int)V, L, false, s));
  NCHECK(net_forward(op, n, w, L, s));
  // column weights 1 / (L ||e_i||^2), loss and delta = d loss / d conj(y)
  double2* npart = reinterpret_cast<double2*>(w->norms);
  double* norm2 = w->norms + 2 * (size_t)PART_STRIDE * NET_BLOCKS;
  NCU(launch_colnorms(static_cast<const double*>(E), L, V * 12, npart, norm2, s));
  wcol_kernel<<<1, 32, 0, s>>>(norm2, w->wcol, L);
  NCU(cudaGetLastError());
  NCU(net_launch_loss_delta(w->act[n->layers], static_cast<const double*>(E), w->wcol, w->dA,
                            w->lpart, NET_BLOCKS, w->loss, (int)V, L, s));
  // backward through the layers
  float* delta = w->dA;
  float* other = w->dB;
  for (int l = n->layers - 1; l >= 0; --l) {
    const int cin = n->ch[l], cout = n->ch[l + 1];
    NCU(net_launch_wgrad(op, w->act[l], delta, cin, cout, L, w->wpart, NET_BLOCKS, n->G + n->off[l], s));
    if (l > 0) {
      NCU(net_launch_adjoint_weights(n->W + n->off[l], n->Wadj + n->off[l], cin, cout, s));
      NCU(net_launch_layer(op, delta, other, n->Wadj + n->off[l], cout, cin, L, s));
      float* t = delta;
      delta = other;
      other = t;
    }
  }
  if (loss) {
    NCU(cudaMemcpyAsync(loss, w->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  if (grad) {
    NCU(cudaMemcpyAsync(grad, n->G, n->nw * sizeof(double2), cudaMemcpyDefault, s));
  }
  NCU(cudaStreamSynchronize(s));
  return WD_OK;
}

int wd_net_adam_step(wd_net* n, double lr, void* stream) {
  if (!n || !(lr > 0.0)) { wd_set_error("net is NULL or lr <= 0"); return WD_EINVAL; }
  n->t += 1;
  NCU(net_launch_adam(n->W, n->G, n->m, n->v, (int)n->nw, (float)lr, 0.9f, 0.999f, 1e-8f, n->t,
                      static_cast<cudaStream_t>(stream)));
  return WD_OK;
}

}  // extern "C"
