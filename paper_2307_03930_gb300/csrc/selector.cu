// Learned schedule selector: problem features, a 3 x 64 ReLU MLP (forward,
// softmax cross-entropy backward, Adam) and its use as a schedule mode.
//
// Sec. 4.2 derives tiles analytically under a uniform-density assumption
// and Sec. 6 leaves auto-tuning open; the selector learns, from the
// autotuner's measured candidate times, which candidate schedule to run for
// a problem's features (sizes, density, row-nonzero histogram, statistics
// of the packed panels).  The analytic rule stays the fallback whenever the
// features fall outside the range the network was trained on.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "handle.hpp"

namespace rosko {

constexpr int kHidden = 64;

namespace {

// ---------------------------------------------------------------------------
// Feature statistics (integer, exact) of a packed handle.
//   s[0] sum row nnz  s[1] sum row nnz^2  s[2] max row nnz
//   s[3..6] rows per density bin (100 r < K | 20 r < K <= 100 r |
//           5 r < K <= 20 r | K <= 5 r)
//   s[7] sum over panels of non-empty columns   s[8] sum panel nnz^2
//   s[9] empty panels
__global__ void row_counts_kernel(const int32_t* __restrict__ panel_col,
                                  const int2* __restrict__ colrec, const void* __restrict__ nz,
                                  rosko_dtype dt, int m_r, int32_t* __restrict__ rowcnt) {
  const int64_t p = blockIdx.x;
  for (int64_t c = panel_col[p] + threadIdx.x; c < panel_col[p + 1]; c += blockDim.x) {
    for (int32_t e = colrec[c].y; e < colrec[c + 1].y; ++e) {
      int r;
      if (dt == ROSKO_F32) r = (int)reinterpret_cast<const uint2*>(nz)[e].x;
      else if (dt == ROSKO_F64) r = reinterpret_cast<const RecF64*>(nz)[e].r;
      else r = (int)(reinterpret_cast<const uint32_t*>(nz)[e] & 0xFFFFu);
      atomicAdd(&rowcnt[p * m_r + r], 1);
    }
  }
}

__global__ void feature_stats_kernel(const int32_t* __restrict__ rowcnt, int64_t M, int64_t K,
                                     const int32_t* __restrict__ panel_col,
                                     const int64_t* __restrict__ panel_nnz, int64_t P,
                                     unsigned long long* __restrict__ s) {
  unsigned long long a[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < M; i += stride) {
    const unsigned long long r = (unsigned long long)rowcnt[i];
    a[0] += r;
    a[1] += r * r;
    a[2] = r > a[2] ? r : a[2];
    const unsigned long long k = (unsigned long long)K;
    if (100 * r < k) a[3]++;
    else if (20 * r < k) a[4]++;
    else if (5 * r < k) a[5]++;
    else a[6]++;
  }
  for (int64_t p = tid; p < P; p += stride) {
    const unsigned long long pn = (unsigned long long)(panel_nnz[p + 1] - panel_nnz[p]);
    a[7] += (unsigned long long)(panel_col[p + 1] - panel_col[p]);
    a[8] += pn * pn;
    a[9] += pn == 0 ? 1 : 0;
  }
  for (int j = 0; j < 10; ++j) {
    if (j == 2) atomicMax(&s[j], a[j]);
    else atomicAdd(&s[j], a[j]);
  }
}

// ---------------------------------------------------------------------------
// MLP kernels (FP32).  Parameters are one flat array, per layer l:
// W_l [out][in] row-major then b_l [out]; sizes 16->64->64->64->C.
struct Layer {
  int in, out;
  int64_t w, b;  // offsets into the parameter array
};

void layers_of(int n_in, int n_out, Layer* L) {
  const int sizes[5] = {n_in, kHidden, kHidden, kHidden, n_out};
  int64_t off = 0;
  for (int l = 0; l < 4; ++l) {
    L[l].in = sizes[l];
    L[l].out = sizes[l + 1];
    L[l].w = off;
    off += (int64_t)sizes[l] * sizes[l + 1];
    L[l].b = off;
    off += sizes[l + 1];
  }
}

// y[b][o] = act(sum_i W[o][i] x[b][i] + bias[o]); relu for hidden layers.
__global__ void dense_forward_kernel(const float* __restrict__ W, const float* __restrict__ bias,
                                     const float* __restrict__ x, int64_t batch, int in, int out,
                                     int relu, float* __restrict__ y) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= batch * out) return;
  const int64_t b = idx / out;
  const int o = (int)(idx % out);
  float acc = bias[o];
  const float* w = W + (int64_t)o * in;
  const float* xb = x + b * in;
  for (int i = 0; i < in; ++i) acc = __fmaf_rn(w[i], xb[i], acc);
  y[idx] = relu ? fmaxf(acc, 0.0f) : acc;
}

// Per sample: loss_b = -sum_c y_c log softmax(z)_c and g = (p sum_c y_c - y) / B.
__global__ void softmax_xent_kernel(const float* __restrict__ z, const float* __restrict__ y,
                                    int64_t batch, int C, float* __restrict__ g,
                                    float* __restrict__ loss) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const float* zb = z + b * C;
  const float* yb = y + b * C;
  float mx = zb[0];
  for (int c = 1; c < C; ++c) mx = fmaxf(mx, zb[c]);
  float se = 0.0f;
  for (int c = 0; c < C; ++c) se += expf(zb[c] - mx);
  const float lse = logf(se);
  float ysum = 0.0f, l = 0.0f;
  for (int c = 0; c < C; ++c) {
    ysum += yb[c];
    l -= yb[c] * (zb[c] - mx - lse);
  }
  for (int c = 0; c < C; ++c) {
    const float p = expf(zb[c] - mx - lse);
    g[b * C + c] = (p * ysum - yb[c]) / (float)batch;
  }
  atomicAdd(loss, l / (float)batch);
}

// dW[o][i] = sum_b g[b][o] x[b][i],  db[o] = sum_b g[b][o]
__global__ void dense_wgrad_kernel(const float* __restrict__ g, const float* __restrict__ x,
                                   int64_t batch, int in, int out, float* __restrict__ dW,
                                   float* __restrict__ db) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)out * (in + 1)) return;
  const int o = (int)(idx / (in + 1));
  const int i = (int)(idx % (in + 1));
  float acc = 0.0f;
  if (i < in) {
    for (int64_t b = 0; b < batch; ++b) acc = __fmaf_rn(g[b * out + o], x[b * in + i], acc);
    dW[(int64_t)o * in + i] = acc;
  } else {
    for (int64_t b = 0; b < batch; ++b) acc += g[b * out + o];
    db[o] = acc;
  }
}

// gx[b][i] = (sum_o W[o][i] g[b][o]) * (x[b][i] > 0)   (x = ReLU output)
__global__ void dense_xgrad_kernel(const float* __restrict__ W, const float* __restrict__ g,
                                   const float* __restrict__ x, int64_t batch, int in, int out,
                                   float* __restrict__ gx) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= batch * in) return;
  const int64_t b = idx / in;
  const int i = (int)(idx % in);
  float acc = 0.0f;
  for (int o = 0; o < out; ++o) acc = __fmaf_rn(W[(int64_t)o * in + i], g[b * out + o], acc);
  gx[idx] = x[idx] > 0.0f ? acc : 0.0f;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2, float wd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i] + wd * p[i];   // gradient of L + (wd / 2) |p|^2
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Selector state loaded by rosko_selector_set.
struct Selector {
  bool set = false;
  int n_out = 0;
  std::vector<float> params;  // host copy
  float* params_dev[64] = {nullptr};
  double mean[kNumFeatures], stdv[kNumFeatures], lo[kNumFeatures], hi[kNumFeatures];
};
Selector g_sel;
std::mutex g_sel_mu;

}  // namespace

int64_t mlp_param_count(int n_in, int n_out) {
  Layer L[4];
  layers_of(n_in, n_out, L);
  return L[3].b + n_out;
}

// Workspace floats for a batch: activations of the 4 layers + gradients.
int64_t mlp_workspace_floats(int64_t batch, int n_out) {
  return batch * (3 * kHidden + n_out) * 2 + 64;
}

rosko_status mlp_forward(const float* params, const float* X, int64_t batch, int n_in, int n_out,
                         float* acts, float* logits, cudaStream_t st) {
  Layer L[4];
  layers_of(n_in, n_out, L);
  const float* in = X;
  for (int l = 0; l < 4; ++l) {
    float* out = (l == 3) ? logits : acts + (int64_t)l * batch * kHidden;
    dense_forward_kernel<<<blocks_for(batch * L[l].out), 256, 0, st>>>(
        params + L[l].w, params + L[l].b, in, batch, L[l].in, L[l].out, l < 3 ? 1 : 0, out);
    in = out;
  }
  count_launches(4);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

rosko_status mlp_loss_grad(const float* params, const float* X, const float* Y, int64_t batch,
                           int n_in, int n_out, float* grads, float* loss, float* ws,
                           cudaStream_t st) {
  Layer L[4];
  layers_of(n_in, n_out, L);
  float* acts = ws;                                   // 3 hidden activations
  float* logits = acts + 3 * batch * kHidden;         // batch x n_out
  float* g_out = logits + batch * n_out;              // dlogits
  float* g_h = g_out + batch * n_out;                 // hidden-layer gradients (3)
  rosko_status s = mlp_forward(params, X, batch, n_in, n_out, acts, logits, st);
  if (s != ROSKO_OK) return s;
  if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return ROSKO_ERR_CUDA;
  softmax_xent_kernel<<<blocks_for(batch), 256, 0, st>>>(logits, Y, batch, n_out, g_out, loss);
  count_launches(1);
  const float* g = g_out;
  for (int l = 3; l >= 0; --l) {
    const float* x_in = (l == 0) ? X : acts + (int64_t)(l - 1) * batch * kHidden;
    dense_wgrad_kernel<<<blocks_for((int64_t)L[l].out * (L[l].in + 1)), 256, 0, st>>>(
        g, x_in, batch, L[l].in, L[l].out, grads + L[l].w, grads + L[l].b);
    count_launches(1);
    if (l > 0) {
      float* gx = g_h + (int64_t)(l - 1) * batch * kHidden;
      dense_xgrad_kernel<<<blocks_for(batch * L[l].in), 256, 0, st>>>(
          params + L[l].w, g, x_in, batch, L[l].in, L[l].out, gx);
      count_launches(1);
      g = gx;
    }
  }
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

rosko_status mlp_adam(float* p, const float* g, float* m, float* v, int64_t n, int step, float lr,
                      float b1, float b2, float eps, float wd, cudaStream_t st) {
  const float c1 = 1.0f - powf(b1, (float)step);
  const float c2 = 1.0f - powf(b2, (float)step);
  adam_kernel<<<blocks_for(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2, wd);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

// The 16 selector features of a handle and width N (definitions in the
// public header).  Integer statistics are reduced on the device; the final
// ratios and logarithms are taken on the host in double.
rosko_status features_impl(rosko_packed_s* h, int64_t N, double* f, cudaStream_t st) {
  const int64_t M = h->M, K = h->K, P = h->P;
  void* scr = nullptr;
  const size_t rc_bytes = ((size_t)std::max<int64_t>(M, 1) * 4 + 255) / 256 * 256;
  if (dev_malloc(&scr, rc_bytes + 256) != cudaSuccess) return ROSKO_ERR_OOM;
  int32_t* rowcnt = static_cast<int32_t*>(scr);
  auto* stats = reinterpret_cast<unsigned long long*>(static_cast<char*>(scr) + rc_bytes);
  rosko_status ret = ROSKO_OK;
  unsigned long long s[10] = {0};
  if (cudaMemsetAsync(scr, 0, rc_bytes + 256, st) != cudaSuccess) ret = ROSKO_ERR_CUDA;
  if (ret == ROSKO_OK && P > 0 && h->nnz > 0) {
    row_counts_kernel<<<(unsigned)P, 128, 0, st>>>(h->panel_col, h->colrec, h->nz, h->dt, h->m_r,
                                                   rowcnt);
    count_launches(1);
  }
  if (ret == ROSKO_OK && M > 0) {
    const unsigned nb = (unsigned)std::min<int64_t>(std::max<int64_t>((M + 255) / 256, 1), 256);
    feature_stats_kernel<<<nb, 256, 0, st>>>(rowcnt, M, K, h->panel_col, h->panel_nnz_dev, P,
                                              stats);
    count_launches(1);
  }
  if (ret == ROSKO_OK &&
      (cudaMemcpyAsync(s, stats, sizeof(s), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    ret = ROSKO_ERR_CUDA;
  cudaFree(scr);
  if (ret != ROSKO_OK) return ret;
  const double Md = (double)M, Kd = (double)K, nnz = (double)s[0];
  const double mean_row = M ? nnz / Md : 0.0;
  f[0] = std::log2(Md);
  f[1] = std::log2(Kd);
  f[2] = std::log2((double)N);
  f[3] = (M && K) ? nnz / (Md * Kd) : 0.0;
  f[4] = std::log2(1.0 + nnz);
  f[5] = std::log2(1.0 + mean_row);
  const double var = M ? (double)s[1] / Md - mean_row * mean_row : 0.0;
  f[6] = mean_row > 0 ? std::sqrt(std::max(var, 0.0)) / mean_row : 0.0;
  f[7] = std::log2(1.0 + (double)s[2]) - std::log2(1.0 + mean_row);
  for (int j = 0; j < 4; ++j) f[8 + j] = M ? (double)s[3 + j] / Md : 0.0;
  const double Pd = (double)P;
  f[12] = (P && K) ? (double)s[7] / (Pd * Kd) : 0.0;
  const double mean_p = P ? nnz / Pd : 0.0;
  const double var_p = P ? (double)s[8] / Pd - mean_p * mean_p : 0.0;
  f[13] = mean_p > 0 ? std::sqrt(std::max(var_p, 0.0)) / mean_p : 0.0;
  f[14] = std::log2(1.0 + (s[7] ? nnz / (double)s[7] : 0.0));
  f[15] = P ? (double)s[9] / Pd : 0.0;
  return ROSKO_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free feature statistics (no counterpart in the paper).
//
// Some callers must not allocate device memory: processes whose device
// memory is handed out by a fixed pool, and latency-critical serving paths
// where cudaMalloc/cudaFree may synchronise the device.  For them the
// feature-statistics kernels above also run on scratch that lives in a
// file-scope device array: every GPU that loads this library holds it
// (4 MiB + 256 B) until the process exits.  Every call shares it and it keeps
// the previous call's contents, so each call clears what must start at zero;
// calls that overlap on the GPU (two streams, two host threads) race on it.
// The largest M served is kStaticRows; larger handles are rejected.
constexpr int64_t kStaticRows = 1 << 20;   // largest M the static scratch serves
static __device__ __align__(256) int32_t g_static_scratch[kStaticRows + 64];

namespace {
// Features from the integer statistics, on the device, in FP32: the same
// definitions as features_impl.  The counts are exact integers; each is
// converted to FP32 once, and the ratios, square roots and logarithms are
// FP32 operations (variances as mean of squares minus squared mean, so a
// small coefficient of variation loses a few bits to cancellation).
__global__ void features_finish_kernel(const unsigned long long* __restrict__ s, int64_t M,
                                       int64_t K, int64_t N, int64_t P, float* __restrict__ out) {
  if (threadIdx.x != 0) return;
  float f[16];
  const float Mf = (float)M, Kf = (float)K, nnz = (float)s[0];
  const float mean_row = M ? nnz / Mf : 0.0f;
  f[0] = log2f(Mf);
  f[1] = log2f(Kf);
  f[2] = log2f((float)N);
  f[3] = (M && K) ? (nnz / Mf) / Kf : 0.0f;
  f[4] = log2f(1.0f + nnz);
  f[5] = log2f(1.0f + mean_row);
  const float var = M ? (float)s[1] / Mf - mean_row * mean_row : 0.0f;
  f[6] = mean_row > 0.0f ? sqrtf(fmaxf(var, 0.0f)) / mean_row : 0.0f;
  f[7] = log2f(1.0f + (float)s[2]) - log2f(1.0f + mean_row);
  for (int j = 0; j < 4; ++j) f[8 + j] = M ? (float)s[3 + j] / Mf : 0.0f;
  const float Pf = (float)P;
  f[12] = (P && K) ? ((float)s[7] / Pf) / Kf : 0.0f;
  const float mean_p = P ? nnz / Pf : 0.0f;
  const float var_p = P ? (float)s[8] / Pf - mean_p * mean_p : 0.0f;
  f[13] = mean_p > 0.0f ? sqrtf(fmaxf(var_p, 0.0f)) / mean_p : 0.0f;
  f[14] = log2f(1.0f + (s[7] ? nnz / (float)s[7] : 0.0f));
  f[15] = P ? (float)s[9] / Pf : 0.0f;
  for (int j = 0; j < 16; ++j) out[j] = f[j];
}
}  // namespace

// Device address of the static scratch on the current device (in host code
// the array's name is only a stand-in).  Looked up with that device current;
// outside a stream capture the lookup is repeated on every call (a host-side
// table lookup), so an address made stale by cudaDeviceReset is never used;
// inside a capture the address cached by the device's last uncaptured call is
// used, which is why the first call on a device must precede any capture.
static int32_t* static_scratch_address(cudaStream_t st) {
  static int32_t* addr[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (cap == cudaStreamCaptureStatusNone || !addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return nullptr;
    addr[dev] = static_cast<int32_t*>(p);
  }
  return addr[dev];
}

rosko_status features_static_impl(rosko_packed_s* h, int64_t N, float* features_dev,
                                  cudaStream_t st) {
  const int64_t M = h->M, K = h->K, P = h->P;
  if (M > kStaticRows) return ROSKO_ERR_INVALID_ARG;
  int32_t* base = static_scratch_address(st);
  if (!base) return ROSKO_ERR_CUDA;
  int32_t* rowcnt = base;
  auto* stats = reinterpret_cast<unsigned long long*>(base + kStaticRows);
  // the previous call's counts are still there: clear rows and statistics
  if ((M > 0 && cudaMemsetAsync(rowcnt, 0, (size_t)M * 4, st) != cudaSuccess) ||
      cudaMemsetAsync(stats, 0, 10 * sizeof(unsigned long long), st) != cudaSuccess)
    return ROSKO_ERR_CUDA;
  if (P > 0 && h->nnz > 0) {
    row_counts_kernel<<<(unsigned)P, 128, 0, st>>>(h->panel_col, h->colrec, h->nz, h->dt, h->m_r,
                                                   rowcnt);
    count_launches(1);
  }
  if (M > 0) {
    const unsigned nb = (unsigned)std::min<int64_t>(std::max<int64_t>((M + 255) / 256, 1), 256);
    feature_stats_kernel<<<nb, 256, 0, st>>>(rowcnt, M, K, h->panel_col, h->panel_nnz_dev, P,
                                              stats);
    count_launches(1);
  }
  features_finish_kernel<<<1, 32, 0, st>>>(stats, M, K, N, P, features_dev);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? ROSKO_OK : ROSKO_ERR_CUDA;
}

rosko_status selector_set(const float* params, int n_params, int n_out, const double* mean,
                          const double* stdv, const double* lo, const double* hi) {
  if (n_out != num_candidates() || n_params != mlp_param_count(kNumFeatures, n_out))
    return ROSKO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_sel_mu);
  g_sel.params.assign(params, params + n_params);
  for (int d = 0; d < 64; ++d) {
    if (g_sel.params_dev[d]) {
      int cur = 0;
      cudaGetDevice(&cur);
      cudaSetDevice(d);
      cudaFree(g_sel.params_dev[d]);
      cudaSetDevice(cur);
      g_sel.params_dev[d] = nullptr;
    }
  }
  for (int j = 0; j < kNumFeatures; ++j) {
    g_sel.mean[j] = mean[j];
    g_sel.stdv[j] = stdv[j] > 0 ? stdv[j] : 1.0;
    g_sel.lo[j] = lo[j];
    g_sel.hi[j] = hi[j];
  }
  g_sel.n_out = n_out;
  g_sel.set = true;
  return ROSKO_OK;
}

rosko_status select_learned(rosko_packed_s* h, int64_t N, rosko_tile* out, cudaStream_t st) {
  std::unique_lock<std::mutex> lk(g_sel_mu);
  if (!g_sel.set) return ROSKO_ERR_UNSUPPORTED;
  lk.unlock();
  double f[kNumFeatures];
  rosko_status s = features_impl(h, N, f, st);
  if (s != ROSKO_OK) return s;
  lk.lock();
  float x[kNumFeatures];
  for (int j = 0; j < kNumFeatures; ++j) {
    // outside the trained range: leave the choice to the analytic rule
    const double span = g_sel.hi[j] - g_sel.lo[j];
    const double slack = 0.05 * span + 1e-9;
    if (f[j] < g_sel.lo[j] - slack || f[j] > g_sel.hi[j] + slack) return ROSKO_ERR_UNSUPPORTED;
    x[j] = (float)((f[j] - g_sel.mean[j]) / g_sel.stdv[j]);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  const int C = g_sel.n_out;
  const int64_t np = (int64_t)g_sel.params.size();
  if (!g_sel.params_dev[dev]) {
    void* pdev = nullptr;
    if (cudaMalloc(&pdev, (size_t)np * 4) != cudaSuccess) return ROSKO_ERR_OOM;
    if (cudaMemcpy(pdev, g_sel.params.data(), (size_t)np * 4, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cudaFree(pdev);
      return ROSKO_ERR_CUDA;
    }
    g_sel.params_dev[dev] = static_cast<float*>(pdev);
  }
  const float* pdev = g_sel.params_dev[dev];
  lk.unlock();
  // one sample through the MLP inference kernels
  void* buf = nullptr;
  const size_t nfl = kNumFeatures + 3 * kHidden + C;
  if (dev_malloc(&buf, nfl * 4) != cudaSuccess) return ROSKO_ERR_OOM;
  float* xin = static_cast<float*>(buf);
  float* acts = xin + kNumFeatures;
  float* logits = acts + 3 * kHidden;
  std::vector<float> z((size_t)C);
  rosko_status r = ROSKO_OK;
  if (cudaMemcpyAsync(xin, x, sizeof(x), cudaMemcpyHostToDevice, st) != cudaSuccess)
    r = ROSKO_ERR_CUDA;
  if (r == ROSKO_OK) r = mlp_forward(pdev, xin, 1, kNumFeatures, C, acts, logits, st);
  if (r == ROSKO_OK && (cudaMemcpyAsync(z.data(), logits, (size_t)C * 4, cudaMemcpyDeviceToHost,
                                        st) != cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
    r = ROSKO_ERR_CUDA;
  cudaFree(buf);
  if (r != ROSKO_OK) return r;
  // argmax over the candidates that apply to this handle
  int best = -1;
  for (int c = 0; c < C; ++c) {
    rosko_tile t;
    if (!candidate_tile(h, N, c, &t)) continue;
    if (best < 0 || z[(size_t)c] > z[(size_t)best]) best = c;
  }
  if (best < 0) return ROSKO_ERR_UNSUPPORTED;
  // The analytic rule stays unless the network prefers another candidate by
  // a clear margin: its logit must exceed that of the candidate matching the
  // rule's schedule by ln 2 (the network rates it at least twice as likely to
  // be the fastest).  Without such a candidate the network decides alone.
  const int eq = analytic_candidate(h, N);
  if (eq >= 0 && eq != best && z[(size_t)best] - z[(size_t)eq] <= 0.6931472f)
    return ROSKO_ERR_UNSUPPORTED;
  if (eq == best) return ROSKO_ERR_UNSUPPORTED;
  candidate_tile(h, N, best, out);
  out->mode = ROSKO_SCHED_FORCED;
  return ROSKO_OK;
}

}  // namespace rosko
