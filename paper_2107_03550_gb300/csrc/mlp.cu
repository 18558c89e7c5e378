// Newton initial-guess network: inference (warp mma.sync, BF16 weights, FP32
// accumulation), training forward/backward and Adam in FP32, all in own
// kernels.  Parameter vector layout (FP32, 4609 + 12): W1[64][5], b1[64],
// W2[64][64], b2[64], W3[64], b3, in_mean[5], in_std[5], out_mean, out_std.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "mlp.cuh"
#include "sbiem.h"

namespace sbiem {

// ----------------------------------------------------------- deployment
__global__ void k_mlp_pack(const float* __restrict__ p, MlpDev* out) {
  const float* W1 = p;
  const float* b1 = W1 + kMlpH * kMlpIn;
  const float* W2 = b1 + kMlpH;
  const float* b2 = W2 + kMlpH * kMlpH;
  const float* W3 = b2 + kMlpH;
  const float* b3 = W3 + kMlpH;
  const float* nrm = b3 + 1;
  for (int i = threadIdx.x; i < kMlpH * 8; i += blockDim.x) {
    const int n = i / 8, j = i % 8;
    const float lo = (2 * j < kMlpIn) ? W1[n * kMlpIn + 2 * j] : 0.f;
    const float hi = (2 * j + 1 < kMlpIn) ? W1[n * kMlpIn + 2 * j + 1] : 0.f;
    out->w1p[n][j] = pack_bf16(lo, hi);
  }
  for (int i = threadIdx.x; i < kMlpH * 32; i += blockDim.x) {
    const int n = i / 32, j = i % 32;
    out->w2p[n][j] = pack_bf16(W2[n * kMlpH + 2 * j], W2[n * kMlpH + 2 * j + 1]);
  }
  for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) {
    out->b1[i] = b1[i];
    out->b2[i] = b2[i];
    out->w3[i] = W3[i];
  }
  if (threadIdx.x == 0) {
    out->b3 = b3[0];
    for (int k = 0; k < kMlpIn; ++k) {
      out->in_mean[k] = nrm[k];
      out->in_std[k] = nrm[kMlpIn + k];
    }
    out->out_mean = nrm[2 * kMlpIn];
    out->out_std = nrm[2 * kMlpIn + 1];
  }
}

// One warp per 32 feature rows (raw features, [n][5]); out[n] = predicted residual.
__global__ void k_mlp_predict(const MlpDev* __restrict__ net, const float* __restrict__ X, int64_t n,
                              float* __restrict__ out) {
  __shared__ MlpDev m;
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(MlpDev) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t*>(&m)[i] = reinterpret_cast<const uint32_t*>(net)[i];
  __syncthreads();
  const int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  float feat[kMlpIn];
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) feat[k] = row < n ? X[row * kMlpIn + k] : m.in_mean[k];
  const float y = mlp_residual_warp(m, feat);
  if (row < n) out[row] = y;
}

// ------------------------------------------------------------- training
constexpr int kTrainRows = 128;  // samples per CTA

// Per-CTA forward / backward of the mean-squared-error loss on normalized
// inputs X[n][5] and targets t[n] (rows idx[b0 .. b0 + B)); writes the CTA's
// partial gradient (scaled by 2/B) and partial loss.
__global__ void __launch_bounds__(kTrainRows) k_mlp_grad(const float* __restrict__ p, const float* __restrict__ X,
                                                          const float* __restrict__ t, const int* __restrict__ idx,
                                                          int64_t b0, int B, float* __restrict__ partial,
                                                          float* __restrict__ loss_partial) {
  extern __shared__ float sm[];
  float* W = sm;                                   // kMlpParams
  float* H1 = W + ((kMlpParams + 31) / 32) * 32;   // [rows][64]: Z1, then GELU(Z1)
  float* H2 = H1 + kTrainRows * kMlpH;             // Z2, then GELU(Z2)
  float* D1 = H2 + kTrainRows * kMlpH;             // dZ1
  float* D2 = D1 + kTrainRows * kMlpH;             // dZ2
  float* dy_s = D2 + kTrainRows * kMlpH;           // [rows]
  float* red = dy_s + kTrainRows;                  // [rows] loss scratch
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) W[i] = p[i];
  __syncthreads();
  const float* W1 = W;
  const float* b1 = W1 + kMlpH * kMlpIn;
  const float* W2 = b1 + kMlpH;
  const float* b2 = W2 + kMlpH * kMlpH;
  const float* W3 = b2 + kMlpH;
  const float b3 = W3[kMlpH];
  const int r = threadIdx.x;
  const int64_t q = b0 + static_cast<int64_t>(blockIdx.x) * kTrainRows + r;
  const bool valid = r < kTrainRows && (q - b0) < B;
  float x[kMlpIn], tt = 0.f;
  if (valid) {
    const int64_t s = idx ? idx[q] : q;
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = X[s * kMlpIn + k];
    tt = t[s];
  } else {
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = 0.f;
  }
  float* h1 = H1 + r * kMlpH;
  float* h2 = H2 + r * kMlpH;
  float* d1 = D1 + r * kMlpH;
  float* d2 = D2 + r * kMlpH;
  // forward: H1 <- Z1, D1 <- GELU(Z1), H2 <- Z2
  for (int j = 0; j < kMlpH; ++j) {
    float z = b1[j];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) z = fmaf(W1[j * kMlpIn + k], x[k], z);
    h1[j] = z;
    d1[j] = gelu_f(z);
  }
  float y = b3;
  for (int j = 0; j < kMlpH; ++j) {
    float z = b2[j];
    for (int k = 0; k < kMlpH; ++k) z = fmaf(W2[j * kMlpH + k], d1[k], z);
    h2[j] = z;
    y = fmaf(W3[j], gelu_f(z), y);
  }
  const float res = valid ? (y - tt) : 0.f;
  const float dy = 2.f * res / static_cast<float>(B);
  dy_s[r] = dy;
  red[r] = res * res;
  // backward: D2 <- dZ2 = dy W3 GELU'(Z2); H2 <- GELU(Z2)
  for (int j = 0; j < kMlpH; ++j) {
    const float z = h2[j];
    const float gp = 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
    d2[j] = dy * W3[j] * gp;
    h2[j] = gelu_f(z);
  }
  // D1 <- dZ1 = (dZ2 W2) GELU'(Z1); H1 <- GELU(Z1) (held in D1 until now)
  for (int k = 0; k < kMlpH; ++k) {
    float s = 0.f;
    for (int j = 0; j < kMlpH; ++j) s = fmaf(d2[j], W2[j * kMlpH + k], s);
    const float z = h1[k];
    const float gp = 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
    const float g1 = d1[k];
    d1[k] = s * gp;
    h1[k] = g1;
  }
  // keep the inputs for dW1
  __shared__ float Xs[kTrainRows][kMlpIn];
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) Xs[r][k] = x[k];
  __syncthreads();
  // partial gradients over this CTA's rows, fixed order
  float* out = partial + static_cast<int64_t>(blockIdx.x) * kMlpParams;
  for (int pi = threadIdx.x; pi < kMlpParams; pi += blockDim.x) {
    float g = 0.f;
    if (pi < kMlpH * kMlpIn) {
      const int j = pi / kMlpIn, k = pi % kMlpIn;
      for (int s = 0; s < kTrainRows; ++s) g = fmaf(D1[s * kMlpH + j], Xs[s][k], g);
    } else if (pi < kMlpH * kMlpIn + kMlpH) {
      const int j = pi - kMlpH * kMlpIn;
      for (int s = 0; s < kTrainRows; ++s) g += D1[s * kMlpH + j];
    } else if (pi < kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH) {
      const int o = pi - (kMlpH * kMlpIn + kMlpH);
      const int j = o / kMlpH, k = o % kMlpH;
      for (int s = 0; s < kTrainRows; ++s) g = fmaf(D2[s * kMlpH + j], H1[s * kMlpH + k], g);
    } else if (pi < kMlpH * kMlpIn + 2 * kMlpH + kMlpH * kMlpH) {
      const int j = pi - (kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH);
      for (int s = 0; s < kTrainRows; ++s) g += D2[s * kMlpH + j];
    } else if (pi < kMlpParams - 1) {
      const int j = pi - (kMlpH * kMlpIn + 2 * kMlpH + kMlpH * kMlpH);
      for (int s = 0; s < kTrainRows; ++s) g = fmaf(dy_s[s], H2[s * kMlpH + j], g);
    } else {
      for (int s = 0; s < kTrainRows; ++s) g += dy_s[s];
    }
    out[pi] = g;
  }
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int s = 0; s < kTrainRows; ++s) l += red[s];
    loss_partial[blockIdx.x] = l;
  }
}

// grad[p] = sum over CTAs of partial[c][p] in CTA order; optional Adam step.
__global__ void k_mlp_reduce(const float* __restrict__ partial, int nblk, float* __restrict__ grad, float* p,
                             float* m1, float* m2, float lr, float beta1, float beta2, float epsa, int step) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= kMlpParams) return;
  float g = 0.f;
  for (int c = 0; c < nblk; ++c) g += partial[static_cast<int64_t>(c) * kMlpParams + pi];
  if (grad) grad[pi] = g;
  if (m1) {
    const float a = beta1 * m1[pi] + (1.f - beta1) * g;
    const float b = beta2 * m2[pi] + (1.f - beta2) * g * g;
    m1[pi] = a;
    m2[pi] = b;
    const float ah = a / (1.f - powf(beta1, static_cast<float>(step)));
    const float bh = b / (1.f - powf(beta2, static_cast<float>(step)));
    p[pi] -= lr * ah / (sqrtf(bh) + epsa);
  }
}

size_t train_smem() {
  return (static_cast<size_t>((kMlpParams + 31) / 32) * 32 + 4 * kTrainRows * kMlpH + 2 * kTrainRows) * sizeof(float);
}

}  // namespace sbiem

using namespace sbiem;

namespace {
thread_local std::string g_mlp_err;
#define MCK(call)                                                   \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) {                                        \
      g_mlp_err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      rc = SBIEM_ERR_CUDA;                                          \
      goto done;                                                    \
    }                                                               \
  } while (0)
}  // namespace

extern "C" {

int sbiem_mlp_predict(const float* params, const float* X, int64_t n, float* out) {
  if (!params || !X || !out || n < 0) return SBIEM_ERR_INVALID;
  int rc = SBIEM_OK;
  float *dp = nullptr, *dX = nullptr, *dout = nullptr;
  MlpDev* net = nullptr;
  MCK(cudaMalloc(&dp, sizeof(float) * (kMlpParams + kMlpNorm)));
  MCK(cudaMalloc(&net, sizeof(MlpDev)));
  MCK(cudaMalloc(&dX, sizeof(float) * kMlpIn * std::max<int64_t>(n, 1)));
  MCK(cudaMalloc(&dout, sizeof(float) * std::max<int64_t>(n, 1)));
  MCK(cudaMemcpy(dp, params, sizeof(float) * (kMlpParams + kMlpNorm), cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(dX, X, sizeof(float) * kMlpIn * n, cudaMemcpyHostToDevice));
  k_mlp_pack<<<1, 256>>>(dp, net);
  if (n > 0) k_mlp_predict<<<static_cast<unsigned>((n + 31) / 32), 32>>>(net, dX, n, dout);
  MCK(cudaGetLastError());
  MCK(cudaMemcpy(out, dout, sizeof(float) * n, cudaMemcpyDeviceToHost));
done:
  cudaFree(dp);
  cudaFree(net);
  cudaFree(dX);
  cudaFree(dout);
  return rc;
}

int sbiem_mlp_grad(const float* params, const float* X, const float* t, int64_t n, float* grad, float* loss) {
  if (!params || !X || !t || !grad || n < 1 || n > (1 << 24)) return SBIEM_ERR_INVALID;
  int rc = SBIEM_OK;
  const int nblk = static_cast<int>((n + kTrainRows - 1) / kTrainRows);
  float *dp = nullptr, *dX = nullptr, *dt = nullptr, *part = nullptr, *lp = nullptr, *dg = nullptr;
  std::vector<float> lh(nblk);
  MCK(cudaMalloc(&dp, sizeof(float) * kMlpParams));
  MCK(cudaMalloc(&dX, sizeof(float) * kMlpIn * n));
  MCK(cudaMalloc(&dt, sizeof(float) * n));
  MCK(cudaMalloc(&part, sizeof(float) * kMlpParams * nblk));
  MCK(cudaMalloc(&lp, sizeof(float) * nblk));
  MCK(cudaMalloc(&dg, sizeof(float) * kMlpParams));
  MCK(cudaMemcpy(dp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(dX, X, sizeof(float) * kMlpIn * n, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(dt, t, sizeof(float) * n, cudaMemcpyHostToDevice));
  MCK(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(train_smem())));
  k_mlp_grad<<<nblk, kTrainRows, train_smem()>>>(dp, dX, dt, nullptr, 0, static_cast<int>(n), part, lp);
  k_mlp_reduce<<<(kMlpParams + 255) / 256, 256>>>(part, nblk, dg, nullptr, nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, 0);
  MCK(cudaGetLastError());
  MCK(cudaMemcpy(grad, dg, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  MCK(cudaMemcpy(lh.data(), lp, sizeof(float) * nblk, cudaMemcpyDeviceToHost));
  if (loss) {
    double l = 0.0;
    for (float v : lh) l += v;
    *loss = static_cast<float>(l / static_cast<double>(n));
  }
done:
  cudaFree(dp);
  cudaFree(dX);
  cudaFree(dt);
  cudaFree(part);
  cudaFree(lp);
  cudaFree(dg);
  return rc;
}

int sbiem_mlp_train(const float* samples, int64_t n, int epochs, int batch, float lr, uint64_t seed,
                    float* params, float* final_loss) {
  // samples: n rows of (ln V_prev, ln theta, tau/sigma, a, b, ln V*)
  if (!samples || !params || n < 2 || epochs < 1 || batch < kTrainRows || !(lr > 0)) return SBIEM_ERR_INVALID;
  int rc = SBIEM_OK;
  // normalization: per-feature mean / std of the inputs and of the residual
  double mean[kMlpIn] = {0}, var[kMlpIn] = {0}, rm = 0.0, rv = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const float* r = samples + i * 6;
    for (int k = 0; k < kMlpIn; ++k) mean[k] += r[k];
    rm += r[5] - r[0];
  }
  for (int k = 0; k < kMlpIn; ++k) mean[k] /= n;
  rm /= n;
  for (int64_t i = 0; i < n; ++i) {
    const float* r = samples + i * 6;
    for (int k = 0; k < kMlpIn; ++k) var[k] += (r[k] - mean[k]) * (r[k] - mean[k]);
    const double d = r[5] - r[0] - rm;
    rv += d * d;
  }
  float in_mean[kMlpIn], in_std[kMlpIn];
  for (int k = 0; k < kMlpIn; ++k) {
    in_mean[k] = static_cast<float>(mean[k]);
    in_std[k] = static_cast<float>(std::max(std::sqrt(var[k] / n), 1e-6));
  }
  const float out_mean = static_cast<float>(rm), out_std = static_cast<float>(std::max(std::sqrt(rv / n), 1e-6));
  std::vector<float> Xn(static_cast<size_t>(n) * kMlpIn), tn(n);
  for (int64_t i = 0; i < n; ++i) {
    const float* r = samples + i * 6;
    for (int k = 0; k < kMlpIn; ++k) Xn[i * kMlpIn + k] = (r[k] - in_mean[k]) / in_std[k];
    tn[i] = (r[5] - r[0] - out_mean) / out_std;
  }
  // He-style initialization (seeded)
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  std::vector<float> p(kMlpParams, 0.f);
  for (int i = 0; i < kMlpH * kMlpIn; ++i) p[i] = nd(rng) * std::sqrt(2.f / kMlpIn);
  for (int i = 0; i < kMlpH * kMlpH; ++i) p[kMlpH * kMlpIn + kMlpH + i] = nd(rng) * std::sqrt(2.f / kMlpH);
  for (int i = 0; i < kMlpH; ++i) p[kMlpH * kMlpIn + 2 * kMlpH + kMlpH * kMlpH + i] = nd(rng) * std::sqrt(1.f / kMlpH);
  const int B = std::min<int64_t>(batch, n);
  const int nblk = (B + kTrainRows - 1) / kTrainRows;
  float *dp = nullptr, *dX = nullptr, *dt = nullptr, *part = nullptr, *lp = nullptr, *m1 = nullptr, *m2 = nullptr;
  int* didx = nullptr;
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  int step = 0;
  double last = 0.0;
  std::vector<float> lh(nblk);
  MCK(cudaMalloc(&dp, sizeof(float) * kMlpParams));
  MCK(cudaMalloc(&m1, sizeof(float) * kMlpParams));
  MCK(cudaMalloc(&m2, sizeof(float) * kMlpParams));
  MCK(cudaMalloc(&dX, sizeof(float) * kMlpIn * n));
  MCK(cudaMalloc(&dt, sizeof(float) * n));
  MCK(cudaMalloc(&didx, sizeof(int) * n));
  MCK(cudaMalloc(&part, sizeof(float) * kMlpParams * nblk));
  MCK(cudaMalloc(&lp, sizeof(float) * nblk));
  MCK(cudaMemcpy(dp, p.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
  MCK(cudaMemset(m1, 0, sizeof(float) * kMlpParams));
  MCK(cudaMemset(m2, 0, sizeof(float) * kMlpParams));
  MCK(cudaMemcpy(dX, Xn.data(), sizeof(float) * kMlpIn * n, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(dt, tn.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
  MCK(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(train_smem())));
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    MCK(cudaMemcpy(didx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    double lsum = 0.0;
    int64_t lcnt = 0;
    for (int64_t b0 = 0; b0 + B <= n; b0 += B) {
      ++step;
      k_mlp_grad<<<nblk, kTrainRows, train_smem()>>>(dp, dX, dt, didx, b0, B, part, lp);
      k_mlp_reduce<<<(kMlpParams + 255) / 256, 256>>>(part, nblk, nullptr, dp, m1, m2, lr, 0.9f, 0.999f, 1e-8f, step);
      if (b0 + 2 * B > n) {  // loss of the epoch's last batch
        MCK(cudaMemcpy(lh.data(), lp, sizeof(float) * nblk, cudaMemcpyDeviceToHost));
        for (float v : lh) lsum += v;
        lcnt += B;
      }
    }
    MCK(cudaGetLastError());
    if (lcnt) last = lsum / static_cast<double>(lcnt);
  }
  MCK(cudaMemcpy(params, dp, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  for (int k = 0; k < kMlpIn; ++k) {
    params[kMlpParams + k] = in_mean[k];
    params[kMlpParams + kMlpIn + k] = in_std[k];
  }
  params[kMlpParams + 2 * kMlpIn] = out_mean;
  params[kMlpParams + 2 * kMlpIn + 1] = out_std;
  if (final_loss) *final_loss = static_cast<float>(last);
done:
  cudaFree(dp);
  cudaFree(m1);
  cudaFree(m2);
  cudaFree(dX);
  cudaFree(dt);
  cudaFree(didx);
  cudaFree(part);
  cudaFree(lp);
  return rc;
}

}  // extern "C"

namespace sbiem {
// Device copy of a deployed network (used by the handle).
int mlp_deploy(const float* params_host, MlpDev* dst, cudaStream_t st) {
  float* dp = nullptr;
  if (cudaMalloc(&dp, sizeof(float) * (kMlpParams + kMlpNorm)) != cudaSuccess) return SBIEM_ERR_NOMEM;
  cudaMemcpyAsync(dp, params_host, sizeof(float) * (kMlpParams + kMlpNorm), cudaMemcpyHostToDevice, st);
  k_mlp_pack<<<1, 256, 0, st>>>(dp, dst);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(dp);
  return e == cudaSuccess ? SBIEM_OK : SBIEM_ERR_CUDA;
}
}  // namespace sbiem
