// MLP cost surrogate: a 3-layer perceptron (in -> hidden -> hidden -> out,
// ReLU) trained with mean squared error and Adam, every step on the device in
// FP32 with the kernels below; plus the C-ABI entry points of the surrogate
// (features, labelled data from the exact counter, training, prediction,
// gradients for checking, and the surrogate-guided cut search).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "../../include/qtn.h"
#include "internal.hpp"
#include "surrogate.hpp"

using namespace qtn;

namespace {

// C[M x N] = op(A)[M x K] * op(B)[K x N] (+ bias[n]) (ReLU), row-major.
// op(A)[m][k] = transA ? A[k * lda + m] : A[m * lda + k]; likewise B.
// 64 x 64 tile per block of 256 threads, 4 x 4 outputs per thread.
constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                   bool transA, const float* __restrict__ B, int ldb, bool transB,
                                                   float* __restrict__ C, int ldc, const float* __restrict__ bias,
                                                   bool relu) {
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int i = threadIdx.x; i < TK * TM; i += 256) {
      const int kk = i / TM, mm = i % TM;
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < K) v = transA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      As[kk][mm] = v;
    }
    for (int i = threadIdx.x; i < TK * TN; i += 256) {
      const int kk = i / TN, nn = i % TN;
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.f;
      if (n < N && k < K) v = transB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
      if (m < M && n < N) {
        float v = acc[i][j];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.f);
        C[(size_t)m * ldc + n] = v;
      }
    }
}

__global__ void relu_backward_kernel(float* __restrict__ dH, const float* __restrict__ H, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (H[i] <= 0.f) dH[i] = 0.f;
}

// db[n] = sum over rows of dY[r][n], one thread per column, rows in order.
__global__ void column_sum_kernel(const float* __restrict__ dY, int rows, int cols, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += dY[(size_t)r * cols + c];
  db[c] = s;
}

// dY = 2 (Y - T) / (rows * cols); per-block partial sums of (Y - T)^2.
__global__ void mse_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                                size_t n, float scale, float* __restrict__ partial) {
  __shared__ float red[256];
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = 2.f * d * scale;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ src, const int* __restrict__ idx, int rows, int cols,
                                   float* __restrict__ dst) {
  const size_t n = (size_t)rows * cols;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[(size_t)idx[i / cols] * cols + i % cols];
}

void gemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, bool tA, const float* B, int ldb, bool tB,
          float* C, int ldc, const float* bias, bool relu) {
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, bias, relu);
}


}  // namespace

struct qtn_mlp {
  int in = 0, hidden = 0, out = 0;
  size_t n_params = 0;
  float* d_params = nullptr;  // W1 b1 W2 b2 W3 b3
  float* d_grads = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  int adam_t = 0;
  std::vector<float> x_mean, x_std, y_mean, y_std;
  // batch workspace
  int cap = 0;
  float *d_X = nullptr, *d_T = nullptr, *d_H1 = nullptr, *d_H2 = nullptr, *d_Y = nullptr;
  float *d_dH1 = nullptr, *d_dH2 = nullptr, *d_dY = nullptr, *d_partial = nullptr;
  std::mutex mu;

  size_t oW1() const { return 0; }
  size_t ob1() const { return oW1() + (size_t)hidden * in; }
  size_t oW2() const { return ob1() + hidden; }
  size_t ob2() const { return oW2() + (size_t)hidden * hidden; }
  size_t oW3() const { return ob2() + hidden; }
  size_t ob3() const { return oW3() + (size_t)out * hidden; }

  ~qtn_mlp() {
    for (float* p : {d_params, d_grads, d_m, d_v, d_X, d_T, d_H1, d_H2, d_Y, d_dH1, d_dH2, d_dY, d_partial})
      cudaFree(p);
  }

  cudaError_t ensure(int n) {
    if (n <= cap) return cudaSuccess;
    for (float** p : {&d_X, &d_T, &d_H1, &d_H2, &d_Y, &d_dH1, &d_dH2, &d_dY}) {
      cudaFree(*p);
      *p = nullptr;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&d_X, sizeof(float) * (size_t)n * in)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_T, sizeof(float) * (size_t)n * out)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_H1, sizeof(float) * (size_t)n * hidden)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_H2, sizeof(float) * (size_t)n * hidden)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_Y, sizeof(float) * (size_t)n * out)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_dH1, sizeof(float) * (size_t)n * hidden)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_dH2, sizeof(float) * (size_t)n * hidden)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_dY, sizeof(float) * (size_t)n * out)) != cudaSuccess) return e;
    cap = n;
    return cudaSuccess;
  }

  void forward(cudaStream_t s, const float* X, int n) {
    const float* P = d_params;
    gemm(s, n, hidden, in, X, in, false, P + oW1(), in, true, d_H1, hidden, P + ob1(), true);
    gemm(s, n, hidden, hidden, d_H1, hidden, false, P + oW2(), hidden, true, d_H2, hidden, P + ob2(), true);
    gemm(s, n, out, hidden, d_H2, hidden, false, P + oW3(), hidden, true, d_Y, out, P + ob3(), false);
  }

  // Gradients of mean((Y - T)^2) over the n x out outputs into d_grads.
  void backward(cudaStream_t s, const float* X, const float* T, int n, int loss_blocks) {
    const size_t ny = (size_t)n * out;
    mse_grad_kernel<<<loss_blocks, 256, 0, s>>>(d_Y, T, d_dY, ny, 1.f / (float)ny, d_partial);
    float* G = d_grads;
    const float* P = d_params;
    // layer 3
    gemm(s, out, hidden, n, d_dY, out, true, d_H2, hidden, false, G + oW3(), hidden, nullptr, false);
    column_sum_kernel<<<(out + 127) / 128, 128, 0, s>>>(d_dY, n, out, G + ob3());
    gemm(s, n, hidden, out, d_dY, out, false, P + oW3(), hidden, false, d_dH2, hidden, nullptr, false);
    relu_backward_kernel<<<256, 256, 0, s>>>(d_dH2, d_H2, (size_t)n * hidden);
    // layer 2
    gemm(s, hidden, hidden, n, d_dH2, hidden, true, d_H1, hidden, false, G + oW2(), hidden, nullptr, false);
    column_sum_kernel<<<(hidden + 127) / 128, 128, 0, s>>>(d_dH2, n, hidden, G + ob2());
    gemm(s, n, hidden, hidden, d_dH2, hidden, false, P + oW2(), hidden, false, d_dH1, hidden, nullptr, false);
    relu_backward_kernel<<<256, 256, 0, s>>>(d_dH1, d_H1, (size_t)n * hidden);
    // layer 1
    gemm(s, hidden, in, n, d_dH1, hidden, true, X, in, false, G + oW1(), in, nullptr, false);
    column_sum_kernel<<<(hidden + 127) / 128, 128, 0, s>>>(d_dH1, n, hidden, G + ob1());
  }

  std::vector<float> normalise_x(const float* X, int n) const {
    std::vector<float> r((size_t)n * in);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < in; ++j) r[(size_t)i * in + j] = (X[(size_t)i * in + j] - x_mean[j]) / x_std[j];
    return r;
  }
  std::vector<float> normalise_y(const float* Y, int n) const {
    std::vector<float> r((size_t)n * out);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < out; ++j) r[(size_t)i * out + j] = (Y[(size_t)i * out + j] - y_mean[j]) / y_std[j];
    return r;
  }

  // Predictions of raw feature rows (host), un-normalised.
  cudaError_t predict(const float* X, int n, float* Y, cudaStream_t s) {
    cudaError_t e = ensure(n);
    if (e != cudaSuccess) return e;
    std::vector<float> xn = normalise_x(X, n);
    if ((e = cudaMemcpyAsync(d_X, xn.data(), xn.size() * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return e;
    forward(s, d_X, n);
    std::vector<float> yn((size_t)n * out);
    if ((e = cudaMemcpyAsync(yn.data(), d_Y, yn.size() * sizeof(float), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < out; ++j) Y[(size_t)i * out + j] = yn[(size_t)i * out + j] * y_std[j] + y_mean[j];
    return cudaGetLastError();
  }
};

namespace {

qtn_status cerr(cudaError_t e, const char* what) {
  return internal::set_error(QTN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define MLP_CUDA(call)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cerr(e_, #call);     \
  } while (0)

}  // namespace

extern "C" {

qtn_status qtn_surrogate_features(const qtn_network_t* net, const int32_t* cuts, int k, float* out) {
  if (!net || !out || k < 0 || (k > 0 && !cuts)) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  const Network* N = internal::network_of(net);
  std::vector<int> c(cuts, cuts + k);
  for (int x : c)
    if (x < 0 || x >= (int)N->indices.size()) return internal::set_error(QTN_ERR_INVALID_ARG, "cut out of range");
  surrogate_features(*N, c, out);
  return QTN_OK;
}

qtn_status qtn_surrogate_labels(const qtn_network_t* net, const int32_t* cuts, int k, float* out) {
  if (!net || !out || k < 0 || (k > 0 && !cuts)) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  const Network* N = internal::network_of(net);
  std::vector<int> c(cuts, cuts + k);
  for (int x : c)
    if (x < 0 || x >= (int)N->indices.size()) return internal::set_error(QTN_ERR_INVALID_ARG, "cut out of range");
  surrogate_labels(*N, c, out);
  return QTN_OK;
}

qtn_status qtn_surrogate_dataset(int count, int n_lo, int n_hi, int p_lo, int p_hi, int k_lo, int k_hi, uint64_t seed,
                                 int threads, float* X, float* Y) {
  if (count < 0 || !X || !Y || n_lo < 4 || n_hi < n_lo || p_lo < 1 || p_hi < p_lo || k_lo < 0 || k_hi < k_lo)
    return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  surrogate_dataset(count, n_lo, n_hi, p_lo, p_hi, k_lo, k_hi, seed, threads, X, Y);
  return QTN_OK;
}

qtn_status qtn_mlp_create(int in, int hidden, int out, uint64_t seed, qtn_mlp_t** res) {
  if (in < 1 || hidden < 1 || out < 1 || !res) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  *res = nullptr;
  qtn_mlp_t* m = new (std::nothrow) qtn_mlp_t;
  if (!m) return internal::set_error(QTN_ERR_OOM, "host allocation failed");
  m->in = in;
  m->hidden = hidden;
  m->out = out;
  m->n_params = m->ob3() + out;
  std::vector<float> p(m->n_params, 0.f);
  std::mt19937_64 g(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  auto init = [&](size_t off, int rows, int cols) {  // He initialisation
    const float sd = std::sqrt(2.f / (float)cols);
    for (size_t i = 0; i < (size_t)rows * cols; ++i) p[off + i] = nd(g) * sd;
  };
  init(m->oW1(), hidden, in);
  init(m->oW2(), hidden, hidden);
  init(m->oW3(), out, hidden);
  m->x_mean.assign(in, 0.f);
  m->x_std.assign(in, 1.f);
  m->y_mean.assign(out, 0.f);
  m->y_std.assign(out, 1.f);
  cudaError_t e = cudaSuccess;
  for (float** d : {&m->d_params, &m->d_grads, &m->d_m, &m->d_v})
    if (e == cudaSuccess) e = cudaMalloc(d, m->n_params * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_partial, 1024 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(m->d_params, p.data(), p.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, m->n_params * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, m->n_params * sizeof(float));
  if (e != cudaSuccess) {
    delete m;
    return cerr(e, "qtn_mlp_create");
  }
  *res = m;
  return QTN_OK;
}

void qtn_mlp_destroy(qtn_mlp_t* m) { delete m; }

qtn_status qtn_mlp_num_params(const qtn_mlp_t* m, size_t* n) {
  if (!m || !n) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  *n = m->n_params;
  return QTN_OK;
}

qtn_status qtn_mlp_params(qtn_mlp_t* m, float* host, int set) {
  if (!m || !host) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(m->mu);
  MLP_CUDA(cudaMemcpy(set ? (void*)m->d_params : (void*)host, set ? (const void*)host : (const void*)m->d_params,
                      m->n_params * sizeof(float), set ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost));
  return QTN_OK;
}

qtn_status qtn_mlp_normalisation(qtn_mlp_t* m, float* x_mean, float* x_std, float* y_mean, float* y_std, int set) {
  if (!m || !x_mean || !x_std || !y_mean || !y_std) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(m->mu);
  if (set) {
    m->x_mean.assign(x_mean, x_mean + m->in);
    m->x_std.assign(x_std, x_std + m->in);
    m->y_mean.assign(y_mean, y_mean + m->out);
    m->y_std.assign(y_std, y_std + m->out);
  } else {
    std::copy(m->x_mean.begin(), m->x_mean.end(), x_mean);
    std::copy(m->x_std.begin(), m->x_std.end(), x_std);
    std::copy(m->y_mean.begin(), m->y_mean.end(), y_mean);
    std::copy(m->y_std.begin(), m->y_std.end(), y_std);
  }
  return QTN_OK;
}

qtn_status qtn_mlp_gradients(qtn_mlp_t* m, const float* X, const float* Y, int n, float* grads, float* loss) {
  if (!m || !X || !Y || n <= 0 || !grads) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(m->mu);
  cudaStream_t s = 0;
  MLP_CUDA(m->ensure(n));
  std::vector<float> xn = m->normalise_x(X, n), yn = m->normalise_y(Y, n);
  MLP_CUDA(cudaMemcpy(m->d_X, xn.data(), xn.size() * sizeof(float), cudaMemcpyHostToDevice));
  MLP_CUDA(cudaMemcpy(m->d_T, yn.data(), yn.size() * sizeof(float), cudaMemcpyHostToDevice));
  m->forward(s, m->d_X, n);
  const int lb = 64;
  m->backward(s, m->d_X, m->d_T, n, lb);
  MLP_CUDA(cudaGetLastError());
  MLP_CUDA(cudaMemcpy(grads, m->d_grads, m->n_params * sizeof(float), cudaMemcpyDeviceToHost));
  if (loss) {
    std::vector<float> part(lb);
    MLP_CUDA(cudaMemcpy(part.data(), m->d_partial, lb * sizeof(float), cudaMemcpyDeviceToHost));
    double t = 0;
    for (float v : part) t += v;
    *loss = (float)(t / ((double)n * m->out));
  }
  return QTN_OK;
}

qtn_status qtn_mlp_fit(qtn_mlp_t* m, const float* X, const float* Y, int n, int epochs, int batch, float lr,
                       uint64_t seed, float* epoch_loss) {
  if (!m || !X || !Y || n <= 0 || epochs < 0 || batch <= 0) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(m->mu);
  // normalisation from the training set
  for (int j = 0; j < m->in; ++j) {
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) {
      s += X[(size_t)i * m->in + j];
      s2 += (double)X[(size_t)i * m->in + j] * X[(size_t)i * m->in + j];
    }
    const double mu = s / n, var = std::max(s2 / n - mu * mu, 0.0);
    m->x_mean[j] = (float)mu;
    m->x_std[j] = var > 1e-12 ? (float)std::sqrt(var) : 1.f;
  }
  for (int j = 0; j < m->out; ++j) {
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) {
      s += Y[(size_t)i * m->out + j];
      s2 += (double)Y[(size_t)i * m->out + j] * Y[(size_t)i * m->out + j];
    }
    const double mu = s / n, var = std::max(s2 / n - mu * mu, 0.0);
    m->y_mean[j] = (float)mu;
    m->y_std[j] = var > 1e-12 ? (float)std::sqrt(var) : 1.f;
  }
  std::vector<float> xn = m->normalise_x(X, n), yn = m->normalise_y(Y, n);
  float *d_allX = nullptr, *d_allY = nullptr;
  int* d_idx = nullptr;
  cudaStream_t s = 0;
  auto cleanup = [&]() {
    cudaFree(d_allX);
    cudaFree(d_allY);
    cudaFree(d_idx);
  };
  cudaError_t e = cudaMalloc(&d_allX, xn.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_allY, yn.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_idx, sizeof(int) * (size_t)batch);
  if (e == cudaSuccess) e = cudaMemcpy(d_allX, xn.data(), xn.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_allY, yn.data(), yn.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = m->ensure(batch);
  if (e != cudaSuccess) {
    cleanup();
    return cerr(e, "qtn_mlp_fit setup");
  }
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::mt19937_64 g(seed);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int lb = 64;
  std::vector<float> part(lb);
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(perm.begin(), perm.end(), g);
    double loss_sum = 0;
    int steps = 0;
    for (int b0 = 0; b0 + batch <= n || (b0 == 0 && n < batch); b0 += batch) {
      const int nb = std::min(batch, n - b0);
      e = cudaMemcpyAsync(d_idx, perm.data() + b0, sizeof(int) * nb, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) break;
      gather_rows_kernel<<<256, 256, 0, s>>>(d_allX, d_idx, nb, m->in, m->d_X);
      gather_rows_kernel<<<64, 256, 0, s>>>(d_allY, d_idx, nb, m->out, m->d_T);
      m->forward(s, m->d_X, nb);
      m->backward(s, m->d_X, m->d_T, nb, lb);
      m->adam_t++;
      const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
      adam_kernel<<<512, 256, 0, s>>>(m->d_params, m->d_grads, m->d_m, m->d_v, m->n_params, lr, b1, b2, eps, c1, c2);
      e = cudaMemcpyAsync(part.data(), m->d_partial, lb * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) break;
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      double t = 0;
      for (float v : part) t += v;
      loss_sum += t / ((double)nb * m->out);
      steps++;
      if (n < batch) break;
    }
    if (e != cudaSuccess) break;
    if (epoch_loss) epoch_loss[ep] = (float)(loss_sum / std::max(steps, 1));
  }
  cleanup();
  if (e != cudaSuccess) return cerr(e, "qtn_mlp_fit");
  return QTN_OK;
}

qtn_status qtn_mlp_predict(qtn_mlp_t* m, const float* X, int n, float* Y) {
  if (!m || !X || !Y || n < 0) return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return QTN_OK;
  std::lock_guard<std::mutex> lk(m->mu);
  MLP_CUDA(m->predict(X, n, Y, 0));
  return QTN_OK;
}

qtn_status qtn_search_cuts_surrogate(const qtn_network_t* net, int k, qtn_mlp_t* m, int T, int N, int top,
                                     uint64_t seed, int seed_greedy, int32_t* cuts, double* best_log2_flops,
                                     int* exact_evals, int* surrogate_evals, double* trace, int trace_cap,
                                     int* trace_len) {
  if (!net || !m || !cuts || k < 1 || T < 0 || N < 2 || top < 1)
    return internal::set_error(QTN_ERR_INVALID_ARG, "bad argument");
  if (m->in != kSurrogateFeatures || m->out != kSurrogateTargets)
    return internal::set_error(QTN_ERR_INVALID_ARG, "surrogate has the wrong input or output width");
  const Network* Nw = internal::network_of(net);
  if (k >= (int)Nw->indices.size()) return internal::set_error(QTN_ERR_INVALID_ARG, "k too large");
  std::lock_guard<std::mutex> lk(m->mu);
  cudaError_t perr = cudaSuccess;
  PredictFn predict = [&](const float* X, int n, float* Y) {
    cudaError_t e = m->predict(X, n, Y, 0);
    if (e != cudaSuccess) perr = e;
  };
  std::vector<std::vector<int>> seeds;
  if (seed_greedy) seeds.push_back(greedy_cuts(*Nw, k));
  SurrogateSearchResult r = surrogate_genetic_cuts(*Nw, k, T, N, top, seed, seeds, predict);
  if (perr != cudaSuccess) return cerr(perr, "surrogate prediction");
  for (int j = 0; j < k; ++j) cuts[j] = r.best[j];
  if (best_log2_flops) *best_log2_flops = r.best_exact;
  if (exact_evals) *exact_evals = r.exact_evaluations;
  if (surrogate_evals) *surrogate_evals = r.surrogate_evaluations;
  int nt = 0;
  if (trace)
    for (; nt < trace_cap && nt < (int)r.best_per_generation.size(); ++nt) trace[nt] = r.best_per_generation[nt];
  if (trace_len) *trace_len = nt;
  return QTN_OK;
}

}  // extern "C"
