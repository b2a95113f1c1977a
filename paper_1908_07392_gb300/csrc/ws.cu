// Learned warm start for the boundary integral equation: a circular 1D convolutional network over
// the boundary nodes with hand-written FP32 forward, backward and Adam kernels.
//
// Layers l = 0..L-1 map C_l -> C_{l+1} channels (C_0 = in_ch, C_L = out_ch, width in between):
//   z_{l+1}[b][o][x] = bias_l[o] + sum_{c,k} W_l[o][c][k] a_l[b][c][(x + k - K/2) mod n],
//   a_{l+1} = relu(z_{l+1}) for l < L-1, output y = z_L.
// Loss mean((y - t)^2); backward: dW_l[o][c][k] = sum_{b,x} dz[b][o][x] a_l[b][c][x + k - K/2],
// dbias_l[o] = sum dz, and da_l = the same convolution of dz with the weights transposed in (o, c)
// and reversed in k; relu masks by a > 0. Adam (Kingma & Ba) with bias correction.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <memory>
#include <new>
#include <vector>

#include "vp_internal.h"
#include "../../include/bie.h"

namespace vp {
namespace {

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

constexpr int kTX = 128;   // positions per block
constexpr int kTO = 16;    // output channels per block
constexpr int kTC = 8;     // input channels per shared chunk
constexpr int kMaxK = 15;

// out[b][o][x] = (bias ? bias[o] : 0) + sum_{c,k} w(o, c, k) in[b][c][(x + k - K/2) mod n]
// with w(o, c, k) = W[o][c][k] (transpose = 0) or W[c][o][K-1-k] (transpose = 1, W of shape [Cin'][Cout'][K]).
__global__ void __launch_bounds__(kTX) k_conv(int n, int Cin, int Cout, int K, int transpose, const float* __restrict__ W,
                                             const float* __restrict__ bias, const float* __restrict__ in,
                                             float* __restrict__ out, int relu) {
  __shared__ float tile[kTC][kTX + kMaxK];
  __shared__ float wsh[kTO][kTC][kMaxK];
  const int x0 = blockIdx.x * kTX, o0 = blockIdx.y * kTO, b = blockIdx.z;
  const int tx = threadIdx.x;
  const int half = K / 2;
  float acc[kTO];
#pragma unroll
  for (int o = 0; o < kTO; ++o) acc[o] = (bias && o0 + o < Cout) ? bias[o0 + o] : 0.f;
  for (int c0 = 0; c0 < Cin; c0 += kTC) {
    for (int e = tx; e < kTC * (kTX + K - 1); e += kTX) {
      const int c = e / (kTX + K - 1), xx = e % (kTX + K - 1);
      int gx = x0 + xx - half;
      gx = ((gx % n) + n) % n;
      tile[c][xx] = (c0 + c < Cin) ? in[((size_t)b * Cin + c0 + c) * n + gx] : 0.f;
    }
    for (int e = tx; e < kTO * kTC * K; e += kTX) {
      const int o = e / (kTC * K), rem = e % (kTC * K), c = rem / K, k = rem % K;
      float v = 0.f;
      if (o0 + o < Cout && c0 + c < Cin) {
        v = transpose ? W[((size_t)(c0 + c) * Cout + (o0 + o)) * K + (K - 1 - k)]
                      : W[((size_t)(o0 + o) * Cin + (c0 + c)) * K + k];
      }
      wsh[o][c][k] = v;
    }
    __syncthreads();
    if (x0 + tx < n) {
      for (int c = 0; c < kTC; ++c)
        for (int k = 0; k < K; ++k) {
          const float v = tile[c][tx + k];
#pragma unroll
          for (int o = 0; o < kTO; ++o) acc[o] = fmaf(wsh[o][c][k], v, acc[o]);
        }
    }
    __syncthreads();
  }
  if (x0 + tx < n) {
#pragma unroll
    for (int o = 0; o < kTO; ++o)
      if (o0 + o < Cout) out[((size_t)b * Cout + o0 + o) * n + x0 + tx] = relu ? fmaxf(acc[o], 0.f) : acc[o];
  }
}

// dW[o][c][k] = sum_{b,x} dz[b][o][x] a[b][c][(x + k - K/2) mod n]; dbias[o] = sum dz (c == 0 blocks).
__global__ void k_conv_wgrad(int n, int B, int Cin, int Cout, int K, const float* __restrict__ dz,
                             const float* __restrict__ a, float* __restrict__ dW, float* __restrict__ dbias) {
  const int o = blockIdx.x, c = blockIdx.y;
  const int half = K / 2;
  float s[kMaxK + 1];
  for (int k = 0; k <= K; ++k) s[k] = 0.f;
  for (int idx = threadIdx.x; idx < B * n; idx += blockDim.x) {
    const int b = idx / n, x = idx % n;
    const float g = dz[((size_t)b * Cout + o) * n + x];
    const float* ar = a + ((size_t)b * Cin + c) * n;
    for (int k = 0; k < K; ++k) {
      int gx = x + k - half;
      gx = gx < 0 ? gx + n : (gx >= n ? gx - n : gx);
      s[k] = fmaf(g, ar[gx], s[k]);
    }
    s[K] += g;
  }
  __shared__ float red[kMaxK + 1][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k <= K; ++k) {
    float v = s[k];
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x <= K) {
    float v = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    if (threadIdx.x < K) dW[((size_t)o * Cin + c) * K + threadIdx.x] = v;
    else if (c == 0) dbias[o] = v;
  }
}

__global__ void k_relu_mask(size_t m, const float* __restrict__ a, float* __restrict__ g) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < m && !(a[i] > 0.f)) g[i] = 0.f;
}

// g = 2 (y - t) / m and partial sums of (y - t)^2 (one per block, into part[blockIdx.x]).
__global__ void k_mse(size_t m, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ g,
                      double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    g[i] = 2.f * d / (float)m;
    s += (double)d * d;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void k_adam(size_t m, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ mo,
                       float* __restrict__ ve, float lr, float b1, float b2, float eps, float c1, float c2) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float gi = g[i];
  const float mi = b1 * mo[i] + (1.f - b1) * gi;
  const float vi = b2 * ve[i] + (1.f - b2) * gi * gi;
  mo[i] = mi;
  ve[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace
}  // namespace vp

struct ws_s {
  int in_ch = 0, width = 0, out_ch = 0, L = 0, K = 0, n = 0, max_batch = 0;
  std::vector<int> C;                       // channels per activation, size L+1
  std::vector<size_t> woff, boff;           // parameter offsets
  size_t nparams = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  std::vector<float*> act;                  // activations a_0..a_{L-1}, z_L (size L+1), max_batch each
  float *d0 = nullptr, *d1 = nullptr;       // gradient work buffers
  double* part = nullptr;
  long long step = 0;
  std::vector<void*> allocs;
};

using namespace vp;

namespace {

int walloc(ws_s* w, float** p, size_t n) {
  void* q = nullptr;
  TRY(cudaMalloc(&q, std::max<size_t>(1, n) * sizeof(float)));
  w->allocs.push_back(q);
  *p = static_cast<float*>(q);
  return VP_OK;
}

// splitmix64 (Steele, Lea and Flood 2014): counter-based seeded uniform numbers for initialisation.
inline uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int forward(ws_s* w, const float* x, int B, cudaStream_t s) {
  const float* in = x;
  for (int l = 0; l < w->L; ++l) {
    const int Cin = w->C[l], Cout = w->C[l + 1];
    float* out = w->act[l + 1];
    dim3 grid((w->n + kTX - 1) / kTX, (Cout + kTO - 1) / kTO, B);
    k_conv<<<grid, kTX, 0, s>>>(w->n, Cin, Cout, w->K, 0, w->p + w->woff[l], w->p + w->boff[l], in, out,
                                l < w->L - 1 ? 1 : 0);
    TRY(cudaGetLastError());
    in = out;
  }
  return VP_OK;
}

int grad(ws_s* w, const float* x, const float* t, int B, float* loss, cudaStream_t s) {
  if (B < 1 || B > w->max_batch) return VP_ERR_ARG;
  // keep the input as a_0 (read only; the caller's buffer)
  int rc = forward(w, x, B, s);
  if (rc) return rc;
  const size_t mout = (size_t)B * w->out_ch * w->n;
  const int nb = 256;
  k_mse<<<nb, 256, 0, s>>>(mout, w->act[w->L], t, w->d0, w->part);
  TRY(cudaGetLastError());
  float* dz = w->d0;
  float* da = w->d1;
  for (int l = w->L - 1; l >= 0; --l) {
    const int Cin = w->C[l], Cout = w->C[l + 1];
    const float* a = (l == 0) ? x : w->act[l];
    k_conv_wgrad<<<dim3(Cout, Cin), 256, 0, s>>>(w->n, B, Cin, Cout, w->K, dz, a, w->g + w->woff[l],
                                                 w->g + w->boff[l]);
    TRY(cudaGetLastError());
    if (l > 0) {
      dim3 grid((w->n + kTX - 1) / kTX, (Cin + kTO - 1) / kTO, B);
      k_conv<<<grid, kTX, 0, s>>>(w->n, Cout, Cin, w->K, 1, w->p + w->woff[l], nullptr, dz, da, 0);
      const size_t ma = (size_t)B * Cin * w->n;
      k_relu_mask<<<(unsigned)((ma + 255) / 256), 256, 0, s>>>(ma, w->act[l], da);
      TRY(cudaGetLastError());
      std::swap(dz, da);
    }
  }
  std::vector<double> part(nb);
  TRY(cudaMemcpyAsync(part.data(), w->part, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  double tot = 0.0;
  for (double v : part) tot += v;
  if (loss) *loss = (float)(tot / (double)mout);
  return VP_OK;
}

}  // namespace

extern "C" void ws_free(ws_net net) {
  if (!net) return;
  for (void* p : net->allocs) cudaFree(p);
  delete net;
}

extern "C" int ws_create(int in_ch, int width, int out_ch, int n_layers, int ksize, int n, int max_batch,
                         uint64_t seed, void* stream, ws_net* out) {
  if (!out) return VP_ERR_ARG;
  *out = nullptr;
  if (in_ch < 1 || width < 1 || out_ch < 1 || n_layers < 1 || ksize < 1 || ksize > kMaxK || (ksize % 2) == 0 ||
      n < ksize || max_batch < 1)
    return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<ws_s> w(new (std::nothrow) ws_s());
  if (!w) return VP_ERR_OOM;
  w->in_ch = in_ch; w->width = width; w->out_ch = out_ch; w->L = n_layers; w->K = ksize; w->n = n;
  w->max_batch = max_batch;
  w->C.assign(n_layers + 1, width);
  w->C[0] = in_ch;
  w->C[n_layers] = out_ch;
  size_t off = 0;
  for (int l = 0; l < n_layers; ++l) {
    w->woff.push_back(off);
    off += (size_t)w->C[l + 1] * w->C[l] * ksize;
    w->boff.push_back(off);
    off += w->C[l + 1];
  }
  w->nparams = off;
  int rc;
  auto fail = [&](int code) { ws_free(w.release()); return code; };
  if ((rc = walloc(w.get(), &w->p, off)) || (rc = walloc(w.get(), &w->g, off)) || (rc = walloc(w.get(), &w->m, off)) ||
      (rc = walloc(w.get(), &w->v, off)))
    return fail(rc);
  w->act.assign(n_layers + 1, nullptr);
  size_t maxc = 0;
  for (int l = 0; l <= n_layers; ++l) maxc = std::max<size_t>(maxc, w->C[l]);
  for (int l = 1; l <= n_layers; ++l)
    if ((rc = walloc(w.get(), &w->act[l], (size_t)max_batch * w->C[l] * n))) return fail(rc);
  if ((rc = walloc(w.get(), &w->d0, (size_t)max_batch * maxc * n)) ||
      (rc = walloc(w.get(), &w->d1, (size_t)max_batch * maxc * n)))
    return fail(rc);
  {
    void* q = nullptr;
    if (cudaMalloc(&q, 256 * sizeof(double)) != cudaSuccess) return fail(VP_ERR_OOM);
    w->allocs.push_back(q);
    w->part = static_cast<double*>(q);
  }
  // initial parameters: uniform in +-1/sqrt(fan_in) from a seeded splitmix64 stream
  std::vector<float> host(off);
  uint64_t st = seed;
  for (int l = 0; l < n_layers; ++l) {
    const float bound = 1.f / std::sqrt((float)(w->C[l] * ksize));
    for (size_t i = w->woff[l]; i < w->boff[l] + w->C[l + 1]; ++i) {
      const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
      host[i] = (float)((2.0 * u - 1.0) * bound);
    }
  }
  if (cudaMemcpyAsync(w->p, host.data(), off * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(w->m, 0, off * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(w->v, 0, off * sizeof(float), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return fail(VP_ERR_CUDA);
  *out = w.release();
  return VP_OK;
}

extern "C" int ws_num_params(ws_net net, int64_t* count) {
  if (!net || !count) return VP_ERR_ARG;
  *count = (int64_t)net->nparams;
  return VP_OK;
}

extern "C" int ws_params(ws_net net, float* buf, int get, void* stream) {
  if (!net || !buf) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (get) TRY(cudaMemcpyAsync(buf, net->p, net->nparams * sizeof(float), cudaMemcpyDeviceToDevice, s));
  else TRY(cudaMemcpyAsync(net->p, buf, net->nparams * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return VP_OK;
}

extern "C" int ws_forward(ws_net net, const float* x, int batch, float* y, void* stream) {
  if (!net || !x || !y || batch < 1 || batch > net->max_batch) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rc = forward(net, x, batch, s);
  if (rc) return rc;
  TRY(cudaMemcpyAsync(y, net->act[net->L], (size_t)batch * net->out_ch * net->n * sizeof(float),
                      cudaMemcpyDeviceToDevice, s));
  return VP_OK;
}

extern "C" int ws_grad(ws_net net, const float* x, const float* t, int batch, float* g, float* loss, void* stream) {
  if (!net || !x || !t || !g) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rc = grad(net, x, t, batch, loss, s);
  if (rc) return rc;
  TRY(cudaMemcpyAsync(g, net->g, net->nparams * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return VP_OK;
}

extern "C" int ws_train_step(ws_net net, const float* x, const float* t, int batch, float lr, float* loss,
                             void* stream) {
  if (!net || !x || !t || !(lr > 0.f)) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rc = grad(net, x, t, batch, loss, s);
  if (rc) return rc;
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
  k_adam<<<(unsigned)((net->nparams + 255) / 256), 256, 0, s>>>(net->nparams, net->p, net->g, net->m, net->v, lr, b1,
                                                                 b2, 1e-8f, c1, c2);
  TRY(cudaGetLastError());
  return VP_OK;
}
