// K8: the capacity predictor's network -- FP32, 1024 -> 64 -> 64 -> 1 with
// ReLU, mapping a sketch's registers (scaled to [0, 1]) to ln(distinct
// vertices).  Forward, backward (mean squared error) and an Adam step, all
// in this file's kernels; no library calls.
//
// Shapes are tiny (a batch of B samples; at most 1024 x 64 weights), so the
// contractions run on CUDA cores with a shared-memory-tiled FP32 GEMM:
// C[m][n] = alpha * sum_k A(m, k) * B(k, n) (+ bias[n]) (+ beta * C) (ReLU),
// where A and B are addressed through (row, column) strides so transposes
// cost nothing.
//
// Parameter layout (DBG_MLP_PARAMS floats): W1 [64][1024] | b1 [64] |
// W2 [64][64] | b2 [64] | w3 [64] | b3 [1].
#include <math.h>

#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

constexpr int kIn = DBG_MLP_INPUTS, kHid = DBG_MLP_HIDDEN;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid;
static_assert(kOffB3 + 1 == DBG_MLP_PARAMS, "parameter layout");

struct Mat {
  const float *p;
  int64_t rs, cs;  // element (r, c) at p[r * rs + c * cs]
  __device__ __forceinline__ float at(int64_t r, int64_t c) const { return p[r * rs + c * cs]; }
};

constexpr int kT = 32;  // tile edge; 16 x 16 threads, 2 x 2 outputs each

// C (M x N, row-major, leading dimension ldc) = alpha * A (M x K) * B (K x N)
// + beta * C + bias[n], then ReLU if asked.
__global__ void __launch_bounds__(256)
    k_gemm(int M, int N, int K, Mat A, Mat B, float *C, int64_t ldc, float alpha, float beta,
           const float *bias, int relu) {
  __shared__ float sa[kT][kT + 1];
  __shared__ float sb[kT][kT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kT, n0 = blockIdx.x * kT;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < K; k0 += kT) {
    for (int i = threadIdx.x; i < kT * kT; i += 256) {
      const int r = i / kT, c = i % kT;
      sa[r][c] = (m0 + r < M && k0 + c < K) ? A.at(m0 + r, k0 + c) : 0.f;
      sb[r][c] = (k0 + r < K && n0 + c < N) ? B.at(k0 + r, n0 + c) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kT; ++kk) {
      const float a0 = sa[ty * 2][kk], a1 = sa[ty * 2 + 1][kk];
      const float b0 = sb[kk][tx * 2], b1 = sb[kk][tx * 2 + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty * 2 + i, n = n0 + tx * 2 + j;
      if (m < M && n < N) {
        float v = alpha * acc[i][j];
        if (beta != 0.f) v += beta * C[(int64_t)m * ldc + n];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.f);
        C[(int64_t)m * ldc + n] = v;
      }
    }
}

int gemm(int M, int N, int K, Mat A, Mat B, float *C, int64_t ldc, float alpha, float beta,
         const float *bias, bool relu, cudaStream_t s) {
  if (M <= 0 || N <= 0) return DBG_OK;
  const dim3 grid((N + kT - 1) / kT, (M + kT - 1) / kT);
  k_gemm<<<grid, 256, 0, s>>>(M, N, K, A, B, C, ldc, alpha, beta, bias, relu ? 1 : 0);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

// dy[i] = (y[i] - t[i]) / B; loss partial sums into *loss (mean squared error / 2).
__global__ void k_loss(const float *y, const float *t, int B, float *dy, float *loss) {
  float part = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = d / (float)B;
    part += 0.5f * d * d / (float)B;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// g[i] *= (h[i] > 0): the ReLU's derivative, in place.
__global__ void k_relu_mask(float *g, const float *h, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (h[i] <= 0.f) g[i] = 0.f;
}

// out[c] = sum_r m[r][c] (column sums of a rows x cols row-major matrix).
__global__ void k_colsum(const float *m, int rows, int cols, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += m[(int64_t)r * cols + c];
  out[c] = s;
}

// Adam (Kingma & Ba 2015) with bias correction, step t >= 1.
__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// He-uniform initial weights from a counter-based hash (SplitMix64 of the
// parameter index), biases zero.
__global__ void k_init(float *p, uint64_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < DBG_MLP_PARAMS;
       i += gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * (1.0f / 16777216.0f) * 2.f - 1.f;  // [-1, 1)
    float v = 0.f;
    if (i < kOffB1) v = u * sqrtf(6.f / kIn);
    else if (i >= kOffW2 && i < kOffB2) v = u * sqrtf(6.f / kHid);
    else if (i >= kOffW3 && i < kOffB3) v = u * sqrtf(6.f / kHid);
    p[i] = v;
  }
}

// x[b][j] = registers[b * stride + j] / 64: sketch registers as network inputs.
__global__ void k_features(const uint32_t *regs, int64_t stride, int B, float *x) {
  const int64_t n = (int64_t)B * kIn;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (float)regs[(i / kIn) * stride + (i % kIn)] * (1.0f / 64.0f);
}

struct Work {
  float *h1, *h2, *y, *dh1, *dh2, *dy, *loss;
};

Work carve(float *w, int B) {
  Work k;
  k.h1 = w;
  k.h2 = k.h1 + (size_t)B * kHid;
  k.dh1 = k.h2 + (size_t)B * kHid;
  k.dh2 = k.dh1 + (size_t)B * kHid;
  k.y = k.dh2 + (size_t)B * kHid;
  k.dy = k.y + B;
  k.loss = k.dy + B;
  return k;
}

int forward(const float *P, const float *x, int B, const Work &w, float *y, cudaStream_t s) {
  int st;
  // H1 = relu(X W1^T + b1)
  st = gemm(B, kHid, kIn, Mat{x, kIn, 1}, Mat{P + kOffW1, 1, kIn}, w.h1, kHid, 1.f, 0.f,
            P + kOffB1, true, s);
  if (st != DBG_OK) return st;
  // H2 = relu(H1 W2^T + b2)
  st = gemm(B, kHid, kHid, Mat{w.h1, kHid, 1}, Mat{P + kOffW2, 1, kHid}, w.h2, kHid, 1.f, 0.f,
            P + kOffB2, true, s);
  if (st != DBG_OK) return st;
  // y = H2 w3 + b3
  return gemm(B, 1, kHid, Mat{w.h2, kHid, 1}, Mat{P + kOffW3, 1, 0}, y, 1, 1.f, 0.f,
              P + kOffB3, false, s);
}

}  // namespace
}  // namespace dbg

using namespace dbg;

extern "C" uint64_t dbg_mlp_work_floats(int batch) {
  return batch <= 0 ? 0 : (uint64_t)batch * (4 * DBG_MLP_HIDDEN + 2) + 1;
}

extern "C" int dbg_mlp_features(const uint32_t *registers, int64_t stride, int batch, float *x,
                                void *stream) {
  if (!registers || !x || batch <= 0 || stride < DBG_MLP_INPUTS) return DBG_ERR_INVALID_ARG;
  k_features<<<256, 256, 0, static_cast<cudaStream_t>(stream)>>>(registers, stride, batch, x);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

extern "C" int dbg_mlp_init(float *params, uint64_t seed, void *stream) {
  if (!params) return DBG_ERR_INVALID_ARG;
  k_init<<<64, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, seed);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

extern "C" int dbg_mlp_forward(const float *params, const float *x, int batch, float *y,
                               float *work, void *stream) {
  if (!params || !x || !y || !work || batch <= 0) return DBG_ERR_INVALID_ARG;
  return forward(params, x, batch, carve(work, batch), y, static_cast<cudaStream_t>(stream));
}

extern "C" int dbg_mlp_train_step(float *params, float *grads, float *adam_m, float *adam_v,
                                  int step, float lr, const float *x, const float *target,
                                  int batch, float *work, float *loss_out, void *stream) {
  if (!params || !grads || !adam_m || !adam_v || !x || !target || !work || batch <= 0 ||
      step < 1 || !(lr > 0.f))
    return DBG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Work w = carve(work, batch);
  float *P = params, *G = grads;
  int st = forward(P, x, batch, w, w.y, s);
  if (st != DBG_OK) return st;
  DBG_CK(cudaMemsetAsync(w.loss, 0, sizeof(float), s));
  k_loss<<<std::max(1, std::min(1024, (batch + 255) / 256)), 256, 0, s>>>(w.y, target, batch,
                                                                          w.dy, w.loss);
  DBG_CK(cudaGetLastError());
  // layer 3: dw3 = H2^T dy, db3 = sum dy, dH2 = (dy w3^T) * relu'(H2)
  st = gemm(kHid, 1, batch, Mat{w.h2, 1, kHid}, Mat{w.dy, 1, 0}, G + kOffW3, 1, 1.f, 0.f,
            nullptr, false, s);
  if (st != DBG_OK) return st;
  k_colsum<<<1, 32, 0, s>>>(w.dy, batch, 1, G + kOffB3);
  st = gemm(batch, kHid, 1, Mat{w.dy, 1, 0}, Mat{P + kOffW3, 0, 1}, w.dh2, kHid, 1.f, 0.f,
            nullptr, false, s);
  if (st != DBG_OK) return st;
  k_relu_mask<<<256, 256, 0, s>>>(w.dh2, w.h2, (int64_t)batch * kHid);
  // layer 2: dW2 = dH2^T H1, db2 = colsum dH2, dH1 = (dH2 W2) * relu'(H1)
  st = gemm(kHid, kHid, batch, Mat{w.dh2, 1, kHid}, Mat{w.h1, kHid, 1}, G + kOffW2, kHid, 1.f,
            0.f, nullptr, false, s);
  if (st != DBG_OK) return st;
  k_colsum<<<(kHid + 63) / 64, 64, 0, s>>>(w.dh2, batch, kHid, G + kOffB2);
  st = gemm(batch, kHid, kHid, Mat{w.dh2, kHid, 1}, Mat{P + kOffW2, kHid, 1}, w.dh1, kHid, 1.f,
            0.f, nullptr, false, s);
  if (st != DBG_OK) return st;
  k_relu_mask<<<256, 256, 0, s>>>(w.dh1, w.h1, (int64_t)batch * kHid);
  // layer 1: dW1 = dH1^T X, db1 = colsum dH1
  st = gemm(kHid, kIn, batch, Mat{w.dh1, 1, kHid}, Mat{x, kIn, 1}, G + kOffW1, kIn, 1.f, 0.f,
            nullptr, false, s);
  if (st != DBG_OK) return st;
  k_colsum<<<(kHid + 63) / 64, 64, 0, s>>>(w.dh1, batch, kHid, G + kOffB1);
  DBG_CK(cudaGetLastError());
  const float b1 = 0.9f, b2 = 0.999f;
  k_adam<<<128, 256, 0, s>>>(P, G, adam_m, adam_v, DBG_MLP_PARAMS, lr, b1, b2, 1e-8f,
                             1.f - powf(b1, (float)step), 1.f - powf(b2, (float)step));
  DBG_CK(cudaGetLastError());
  if (loss_out) DBG_CK(cudaMemcpyAsync(loss_out, w.loss, sizeof(float), cudaMemcpyDefault, s));
  return DBG_OK;
}
