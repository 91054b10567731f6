// C-ABI of the learned period proposal's network (declared in include/qlp_bls.h):
// a 6-layer 1-D CNN over the coarse spectrum's QLP_CNN_IN_CH channels (S/N, valid
// mask, S/N at the bins of 2P, P/2, 3P and P/3):
//   conv(6->64)+ReLU, 4 x [conv(64->64)+ReLU], conv(64->1) -> one logit per bin,
// kernel 9, same padding. Parameters are FP32 masters (Adam); the 64->64 layers
// run on the tensor cores from BF16 copies repacked after every update.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qlp_internal.h"

namespace qlp {
int launch_conv_in(const void* x0, const float* w1, const float* b1, void* a1, int batch, int len, void* s);
int launch_conv_out(const void* a5, const float* w6, const float* b6, float* logit, int batch, int len, void* s);
int launch_bce(const float* logit, const float* label, float* dlogit, float* loss, int n, float pw, void* s);
int launch_conv_out_bwd(const float* dlogit, const float* w6, const void* a5, void* da5, int batch, int len,
                        void* s);
int launch_wgrad64(const void* dy, const void* x, float* partial, float* out, int32_t* err, int batch, int len,
                   void* s);
int launch_dw_small(const void* dy, int dy_is_f32, const void* x, float* partial, float* out, int batch,
                    int len, int n_co, int n_ci, void* s);
int launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float omb1,
                float omb2, float eps, float c1, float c2, void* s);
int wgrad64_parts(int batch, int len);
int dw_small_parts(int batch, int len);
}  // namespace qlp

using namespace qlp;

namespace {

constexpr int kCh = 64, kK = 9, kIn = QLP_CNN_IN_CH;
constexpr int kW1 = kK * kCh * kIn, kW64 = kK * kCh * kCh, kW6 = kK * kCh;
// parameter offsets: [W1 | b1 | (W_k | b_k) k = 2..5 | W6 | b6]
constexpr int kOffW1 = 0, kOffB1 = kW1;
constexpr int off_w(int k) { return kW1 + kCh + (k - 2) * (kW64 + kCh); }  // k = 2..5
constexpr int kOffW6 = kW1 + kCh + 4 * (kW64 + kCh);
constexpr int kOffB6 = kOffW6 + kW6;
constexpr int kNParams = kOffB6 + 1;
constexpr size_t kPackBytes = 73728;

thread_local std::string g_err;

int fail(cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  g_err = buf;
  return QLP_ERR_CUDA;
}
#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return fail(e_, #call);    \
  } while (0)
#define CKL(x)                                                      \
  do {                                                              \
    int e_ = (x);                                                   \
    if (e_) return fail((cudaError_t)e_, #x);                       \
  } while (0)

// splitmix64 counter-based generator and Box-Muller normals for the initial weights
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
double unit01(uint64_t& s) { return ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
double normal(uint64_t& s) {
  const double u = unit01(s), v = unit01(s);
  return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * v);
}

}  // namespace

struct qlp_cnn {
  int max_batch = 0, len = 0;
  int64_t step = 0;
  float* params = nullptr;
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  void* pack_f[4] = {};
  void* pack_b[4] = {};
  void* act[6] = {};   // act[1..5]: layer outputs, BF16 [B][L][64]
  void* gact[6] = {};  // gact[1..5]: gradients w.r.t. pre-activations, BF16 [B][L][64]
  float* logit = nullptr;
  float* dlogit = nullptr;
  float* loss = nullptr;
  int32_t* err = nullptr;
  float* partial = nullptr;
  size_t held = 0;  // device bytes held against the library's budget
};
typedef struct qlp_cnn qlp_cnn_t;

static void cnn_free(qlp_cnn_t* n) {
  if (!n) return;
  cudaFree(n->params); cudaFree(n->grads); cudaFree(n->m); cudaFree(n->v);
  for (int i = 0; i < 4; ++i) { cudaFree(n->pack_f[i]); cudaFree(n->pack_b[i]); }
  for (int i = 0; i < 6; ++i) { cudaFree(n->act[i]); cudaFree(n->gact[i]); }
  cudaFree(n->logit); cudaFree(n->dlogit); cudaFree(n->loss); cudaFree(n->err); cudaFree(n->partial);
  budget_give(n->held);
  delete n;
}

static int repack(qlp_cnn_t* n, void* stream) {
  for (int k = 2; k <= 5; ++k) {
    CKL(launch_pack_w64(n->params + off_w(k), n->pack_f[k - 2], 0, stream));
    CKL(launch_pack_w64(n->params + off_w(k), n->pack_b[k - 2], 1, stream));
  }
  return QLP_OK;
}

extern "C" {

int32_t qlp_cnn_n_params(void) { return kNParams; }

const char* qlp_cnn_last_error(void) { return g_err.c_str(); }

int qlp_cnn_create(int32_t max_batch, int32_t len, uint64_t seed, qlp_cnn_t** out) {
  if (!out || max_batch <= 0 || len <= 0 || len % 128 != 0) return QLP_ERR_ARG;
  *out = nullptr;
  qlp_cnn_t* n = new (std::nothrow) qlp_cnn_t();
  if (!n) return QLP_ERR_NOMEM;
  n->max_batch = max_batch;
  n->len = len;
  const size_t pos = (size_t)max_batch * len;
  const size_t parts = std::max((size_t)wgrad64_parts(max_batch, len) * (kW64 + kCh),
                                (size_t)dw_small_parts(max_batch, len) * (kW1 + kCh));
  const size_t total = sizeof(float) * (4 * (size_t)kNParams + 2 * pos + parts + 1) + sizeof(int32_t) +
                       8 * kPackBytes + 10 * pos * kCh * 2;
  if (!budget_take(total)) {
    delete n;
    return QLP_ERR_NOMEM;
  }
  n->held = total;
  bool ok = cudaMalloc(&n->params, sizeof(float) * kNParams) == cudaSuccess &&
            cudaMalloc(&n->grads, sizeof(float) * kNParams) == cudaSuccess &&
            cudaMalloc(&n->m, sizeof(float) * kNParams) == cudaSuccess &&
            cudaMalloc(&n->v, sizeof(float) * kNParams) == cudaSuccess &&
            cudaMalloc(&n->logit, sizeof(float) * pos) == cudaSuccess &&
            cudaMalloc(&n->dlogit, sizeof(float) * pos) == cudaSuccess &&
            cudaMalloc(&n->loss, sizeof(float)) == cudaSuccess &&
            cudaMalloc(&n->err, sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&n->partial, sizeof(float) * parts) == cudaSuccess;
  for (int i = 0; ok && i < 4; ++i)
    ok = cudaMalloc(&n->pack_f[i], kPackBytes) == cudaSuccess && cudaMalloc(&n->pack_b[i], kPackBytes) == cudaSuccess;
  for (int i = 1; ok && i <= 5; ++i)
    ok = cudaMalloc(&n->act[i], pos * kCh * 2) == cudaSuccess && cudaMalloc(&n->gact[i], pos * kCh * 2) == cudaSuccess;
  if (!ok) {
    cnn_free(n);
    return QLP_ERR_NOMEM;
  }
  // He-normal initial weights (std sqrt(2 / fan_in)), zero biases; the output bias
  // starts at -4 (a prior of ~2 % positives)
  std::vector<float> h(kNParams, 0.f);
  uint64_t st = seed * 0x9e3779b97f4a7c15ull + 12345;
  for (int i = 0; i < kW1; ++i) h[kOffW1 + i] = (float)(normal(st) * std::sqrt(2.0 / (kK * kIn)));
  for (int k = 2; k <= 5; ++k)
    for (int i = 0; i < kW64; ++i) h[off_w(k) + i] = (float)(normal(st) * std::sqrt(2.0 / (kK * kCh)));
  for (int i = 0; i < kW6; ++i) h[kOffW6 + i] = (float)(normal(st) * std::sqrt(1.0 / (kK * kCh)));
  h[kOffB6] = -4.f;
  if (cudaMemcpy(n->params, h.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->m, 0, sizeof(float) * kNParams) != cudaSuccess ||
      cudaMemset(n->v, 0, sizeof(float) * kNParams) != cudaSuccess ||
      cudaMemset(n->grads, 0, sizeof(float) * kNParams) != cudaSuccess ||
      cudaMemset(n->err, 0, sizeof(int32_t)) != cudaSuccess || repack(n, nullptr) != QLP_OK ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cnn_free(n);
    return QLP_ERR_CUDA;
  }
  *out = n;
  return QLP_OK;
}

void qlp_cnn_destroy(qlp_cnn_t* n) { cnn_free(n); }

int qlp_cnn_set_params(qlp_cnn_t* n, const float* host, void* stream) {
  if (!n || !host) return QLP_ERR_ARG;
  CK(cudaMemcpyAsync(n->params, host, sizeof(float) * kNParams, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  CK(cudaMemsetAsync(n->m, 0, sizeof(float) * kNParams, (cudaStream_t)stream));
  CK(cudaMemsetAsync(n->v, 0, sizeof(float) * kNParams, (cudaStream_t)stream));
  n->step = 0;
  const int rc = repack(n, stream);
  if (rc) return rc;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return QLP_OK;
}

int qlp_cnn_get_tensor(const qlp_cnn_t* n, int32_t which, int32_t layer, int32_t batch, void* host,
                       int64_t bytes, void* stream) {
  if (!n || !host || batch <= 0 || batch > n->max_batch) return QLP_ERR_ARG;
  const size_t pos = (size_t)batch * (size_t)n->len;
  const void* src = nullptr;
  size_t need = 0;
  if (which == QLP_CNN_ACT || which == QLP_CNN_GACT) {
    if (layer < 1 || layer > 5) return QLP_ERR_ARG;
    src = which == QLP_CNN_ACT ? n->act[layer] : n->gact[layer];
    need = pos * kCh * 2;
  } else if (which == QLP_CNN_LOGIT || which == QLP_CNN_DLOGIT) {
    src = which == QLP_CNN_LOGIT ? n->logit : n->dlogit;
    need = pos * sizeof(float);
  } else {
    return QLP_ERR_ARG;
  }
  if (bytes < (int64_t)need) return QLP_ERR_ARG;
  CK(cudaMemcpyAsync(host, src, need, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return QLP_OK;
}

int qlp_cnn_shape(const qlp_cnn_t* n, int32_t* max_batch, int32_t* len) {
  if (!n) return QLP_ERR_ARG;
  if (max_batch) *max_batch = n->max_batch;
  if (len) *len = n->len;
  return QLP_OK;
}

// Checkpoint file: 8-byte tag, int32 parameter count, int32 zero, int64 Adam step,
// then the FP32 parameters, Adam's first and second moments (little-endian).
static const char kTag[8] = {'Q', 'L', 'P', 'C', 'N', 'N', '0', '1'};

int qlp_cnn_save(const qlp_cnn_t* n, const char* path, void* stream) {
  if (!n || !path) return QLP_ERR_ARG;
  std::vector<float> buf((size_t)kNParams * 3);
  CK(cudaMemcpyAsync(buf.data(), n->params, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaMemcpyAsync(buf.data() + kNParams, n->m, sizeof(float) * kNParams, cudaMemcpyDeviceToHost,
                     (cudaStream_t)stream));
  CK(cudaMemcpyAsync(buf.data() + 2 * (size_t)kNParams, n->v, sizeof(float) * kNParams, cudaMemcpyDeviceToHost,
                     (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) { g_err = std::string("cannot open ") + path; return QLP_ERR_ARG; }
  const int32_t hdr[2] = {kNParams, 0};
  const int64_t step = n->step;
  bool ok = std::fwrite(kTag, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            std::fwrite(&step, sizeof(step), 1, f) == 1 &&
            std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) { g_err = std::string("write failed: ") + path; return QLP_ERR_ARG; }
  return QLP_OK;
}

int qlp_cnn_load(qlp_cnn_t* n, const char* path, void* stream) {
  if (!n || !path) return QLP_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) { g_err = std::string("cannot open ") + path; return QLP_ERR_ARG; }
  char tag[8];
  int32_t hdr[2];
  int64_t step = 0;
  std::vector<float> buf((size_t)kNParams * 3);
  bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, kTag, 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kNParams &&
            std::fread(&step, sizeof(step), 1, f) == 1 && step >= 0 &&
            std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) { g_err = std::string("not a checkpoint of this network: ") + path; return QLP_ERR_ARG; }
  CK(cudaMemcpyAsync(n->params, buf.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  CK(cudaMemcpyAsync(n->m, buf.data() + kNParams, sizeof(float) * kNParams, cudaMemcpyHostToDevice,
                     (cudaStream_t)stream));
  CK(cudaMemcpyAsync(n->v, buf.data() + 2 * (size_t)kNParams, sizeof(float) * kNParams, cudaMemcpyHostToDevice,
                     (cudaStream_t)stream));
  n->step = step;
  const int rc = repack(n, stream);
  if (rc) return rc;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return QLP_OK;
}

int qlp_cnn_get_params(const qlp_cnn_t* n, float* host, float* grads_host, void* stream) {
  if (!n) return QLP_ERR_ARG;
  if (host) CK(cudaMemcpyAsync(host, n->params, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  if (grads_host)
    CK(cudaMemcpyAsync(grads_host, n->grads, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return QLP_OK;
}

int qlp_cnn_forward(qlp_cnn_t* n, const void* x0, int32_t batch, float* logits, void* stream) {
  if (!n || !x0 || batch <= 0 || batch > n->max_batch) return QLP_ERR_ARG;
  const int L = n->len;
  CKL(launch_conv_in(x0, n->params + kOffW1, n->params + kOffB1, n->act[1], batch, L, stream));
  for (int k = 2; k <= 5; ++k)
    CKL(launch_conv64(n->act[k - 1], n->pack_f[k - 2], n->params + off_w(k) + kW64, nullptr, n->act[k], n->err,
                      batch, L, 1, stream));
  CKL(launch_conv_out(n->act[5], n->params + kOffW6, n->params + kOffB6, n->logit, batch, L, stream));
  if (logits)
    CK(cudaMemcpyAsync(logits, n->logit, sizeof(float) * (size_t)batch * L, cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
  return QLP_OK;
}

int qlp_cnn_backward(qlp_cnn_t* n, const void* x0, const float* labels, int32_t batch, float pos_weight,
                     void* stream) {
  if (!n || !x0 || !labels || batch <= 0 || batch > n->max_batch) return QLP_ERR_ARG;
  const int L = n->len;
  int rc = qlp_cnn_forward(n, x0, batch, nullptr, stream);
  if (rc) return rc;
  CK(cudaMemsetAsync(n->loss, 0, sizeof(float), (cudaStream_t)stream));
  CKL(launch_bce(n->logit, labels, n->dlogit, n->loss, batch * L, pos_weight, stream));
  CKL(launch_dw_small(n->dlogit, 1, n->act[5], n->partial, n->grads + kOffW6, batch, L, 1, kCh, stream));
  CKL(launch_conv_out_bwd(n->dlogit, n->params + kOffW6, n->act[5], n->gact[5], batch, L, stream));
  for (int k = 5; k >= 2; --k) {
    CKL(launch_wgrad64(n->gact[k], n->act[k - 1], n->partial, n->grads + off_w(k), n->err, batch, L, stream));
    CKL(launch_conv64(n->gact[k], n->pack_b[k - 2], nullptr, n->act[k - 1], n->gact[k - 1], n->err, batch, L, 0,
                      stream));
  }
  CKL(launch_dw_small(n->gact[1], 0, x0, n->partial, n->grads + kOffW1, batch, L, kCh, kIn, stream));
  return QLP_OK;
}

int qlp_cnn_adam_step(qlp_cnn_t* n, float lr, void* stream) {
  if (!n) return QLP_ERR_ARG;
  n->step += 1;
  // beta1 = 0.9, beta2 = 0.999: the complements and the bias corrections in FP64,
  // each rounded once to FP32
  const double b1 = 0.9, b2 = 0.999;
  const double c1 = 1.0 - std::pow(b1, (double)n->step), c2 = 1.0 - std::pow(b2, (double)n->step);
  CKL(launch_adam(n->params, n->grads, n->m, n->v, kNParams, lr, (float)b1, (float)b2, (float)(1.0 - b1),
                  (float)(1.0 - b2), 1e-8f, (float)c1, (float)c2, stream));
  return repack(n, stream);
}

int qlp_cnn_train_step(qlp_cnn_t* n, const void* x0, const float* labels, int32_t batch, float pos_weight,
                       float lr, void* stream) {
  int rc = qlp_cnn_backward(n, x0, labels, batch, pos_weight, stream);
  if (rc) return rc;
  return qlp_cnn_adam_step(n, lr, stream);
}

int qlp_cnn_loss(qlp_cnn_t* n, float* loss_host, int32_t* err_host, void* stream) {
  if (!n) return QLP_ERR_ARG;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (loss_host) CK(cudaMemcpy(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost));
  int32_t e = 0;
  CK(cudaMemcpy(&e, n->err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (err_host) *err_host = e;
  return e ? QLP_ERR_DEVICE : QLP_OK;
}

int64_t qlp_cnn_wgrad64_workspace(int32_t batch, int32_t len) {
  if (batch <= 0 || len <= 0 || len % 128 != 0) return 0;
  return (int64_t)wgrad64_parts(batch, len) * (kW64 + kCh);
}

int qlp_cnn_conv64_wgrad(const void* dy, const void* x, float* workspace, float* out, int32_t batch, int32_t len,
                         int32_t* err, void* stream) {
  if (!dy || !x || !workspace || !out || !err || batch <= 0 || len <= 0 || len % 128 != 0) return QLP_ERR_ARG;
  CKL(launch_wgrad64(dy, x, workspace, out, err, batch, len, stream));
  return QLP_OK;
}

int qlp_cnn_pack_w64(const float* w, void* wpack, int32_t transpose, void* stream) {
  if (!w || !wpack || (reinterpret_cast<uintptr_t>(wpack) & 15u) != 0) return QLP_ERR_ARG;
  CKL(launch_pack_w64(w, wpack, transpose, stream));
  return QLP_OK;
}

int qlp_cnn_conv64(const void* x, const void* wpack, const float* bias, const void* mask, void* y,
                   int32_t batch, int32_t len, int32_t relu, int32_t* err, void* stream) {
  // the weights arrive by one bulk copy and the activations by TMA: 16-byte boundaries
  if (!x || !wpack || !y || !err || batch < 0 || len <= 0 || len % 128 != 0 ||
      ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(wpack) | reinterpret_cast<uintptr_t>(y)) & 15u) != 0)
    return QLP_ERR_ARG;
  CKL(launch_conv64(x, wpack, bias, mask, y, err, batch, len, relu, stream));
  return QLP_OK;
}

}  // extern "C"
