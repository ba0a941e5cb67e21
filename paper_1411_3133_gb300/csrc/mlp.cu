// Surrogate of developed channel flow: a multilayer perceptron mapping
// channel parameters (Dean number, curvature ratio, ...) and a node's
// position to the macroscopic fields (rho', u^r, u^theta, u^3) of a
// converged LB run, used to warm-start the LB (lb_init_fields). Hand-written
// kernels for the forward pass, the backward pass and the Adam update;
// weights are kept in FP32 (master copy, Adam moments) and used in BF16 by
// every product, which accumulates in FP32.
//
// Layers: features phi(x) = (p_1 .. p_P, sin(2 pi k z), cos(2 pi k z), k =
// 1..F) of an input row (p_1 .. p_P, z),
// then depth - 1 hidden layers of `width` units with SiLU, then a linear
// output layer of 4 units. Outputs are normalised per field: the network
// predicts (y - mean) / std.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbgm.h"

namespace {

constexpr int NOUT = 4;

// --------------------------------------------------------------------------
// kernels
// --------------------------------------------------------------------------
// Row i of x holds np plain inputs then z; its features are the plain
// inputs then sin(2 pi k z), cos(2 pi k z), k = 1..nf.
__global__ void k_features(const float* __restrict__ x, int n, int np, int nf, float* __restrict__ phi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nin = np + 2 * nf;
  const float* xi = x + size_t(i) * (np + 1);
  float* o = phi + size_t(i) * nin;
  for (int j = 0; j < np; ++j) o[j] = xi[j];
  const float z = xi[np];
  for (int k = 1; k <= nf; ++k) {
    float s, c;
    sincospif(2.0f * float(k) * z, &s, &c);
    o[np + 2 * k - 2] = s;
    o[np + 2 * k - 1] = c;
  }
}

template <class T>
__device__ __forceinline__ float ldf(const T* p) { return float(*p); }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[m][n] = sum_k A(m, k) B(k, n) (+ C[m][n] if accumulate), FP32
// accumulation; A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn].
// 64 x 64 output tiles, 16-deep k slices staged in shared memory, 256
// threads with 4 x 4 outputs each.
constexpr int TM = 64, TN = 64, TK = 16;
template <class TA, class TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const TA* __restrict__ A, long sam, long sak,
                                              const TB* __restrict__ B, long sbk, long sbn, float* __restrict__ C,
                                              int ldc, int accumulate) {
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      const int kk = e / TM, mm = e % TM;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? ldf(A + m * sam + k * sak) : 0.0f;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      const int kk = e / TN, nn = e % TN;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K) ? ldf(B + k * sbk + n * sbn) : 0.0f;
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
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float* c = C + size_t(m) * ldc + n;
      *c = accumulate ? *c + acc[i][j] : acc[i][j];
    }
  }
}

__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

// Z += bias (per column); H = SiLU(Z) when act, else H = Z.
__global__ void k_bias_act(float* __restrict__ Z, float* __restrict__ H, const float* __restrict__ bias, int n,
                           int width, int act) {
  const size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (i >= size_t(n) * width) return;
  const float z = Z[i] + bias[i % width];
  Z[i] = z;
  H[i] = act ? z * sigmoidf(z) : z;
}

// dZ = dH * SiLU'(Z)
__global__ void k_silu_back(const float* __restrict__ Z, float* __restrict__ dZ, size_t count) {
  const size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (i >= count) return;
  const float s = sigmoidf(Z[i]);
  dZ[i] *= s * (1.0f + Z[i] * (1.0f - s));
}

// Mean squared error of normalised outputs: dY = 2 (Y - T) / (n NOUT),
// T = (y - mean) / std; per-block partial sums of the squared error.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ y, const float* __restrict__ mean,
                      const float* __restrict__ istd, int n, float* __restrict__ dY, float* __restrict__ partial) {
  __shared__ float sh[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float e2 = 0.0f;
  if (i < n * NOUT) {
    const int q = i % NOUT;
    const float t = (y[i] - mean[q]) * istd[q];
    const float d = Y[i] - t;
    dY[i] = 2.0f * d / float(n * NOUT);
    e2 = d * d;
  }
  sh[threadIdx.x] = e2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum(const float* __restrict__ partial, int n, float denom, float* __restrict__ out) {
  __shared__ float sh[256];
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] / denom;
}

// db[j] = sum_i dZ[i][j]
__global__ void k_colsum(const float* __restrict__ dZ, int n, int width, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= width) return;
  float s = 0.0f;
  for (int i = 0; i < n; ++i) s += dZ[size_t(i) * width + j];
  db[j] = s;
}

// Adam on the FP32 master parameters; refreshes their BF16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, size_t count, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
  const size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, size_t count) {
  const size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (i < count) wb[i] = __float2bfloat16_rn(w[i]);
}

// y = Y * std + mean
__global__ void k_denorm(const float* __restrict__ Y, const float* __restrict__ mean, const float* __restrict__ sd,
                         int n, float* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * NOUT) y[i] = Y[i] * sd[i % NOUT] + mean[i % NOUT];
}

unsigned nblk(size_t n, int t = 256) { return unsigned((n + t - 1) / t); }

}  // namespace

struct lb_mlp {
  int np = 0, nf = 0, width = 0, depth = 0, max_batch = 0, nin = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> fan_in, fan_out;       // per layer
  std::vector<size_t> w_off, b_off;       // offsets into the parameter arrays
  size_t nparam = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* wb = nullptr;
  float *phi = nullptr, *dY = nullptr, *Yout = nullptr, *partial = nullptr, *loss = nullptr;
  std::vector<float*> Z, H;                // per hidden layer [max_batch][width]
  float *dA = nullptr, *dB = nullptr;      // gradient scratch [max_batch][width]
  float* scale = nullptr;                  // mean[4], istd[4], std[4]
  long long steps = 0;
  std::string err;
  std::vector<void*> allocs;
};

namespace {

thread_local std::string g_mlp_err;

lb_status mfail(lb_mlp* n, lb_status s, const std::string& msg) {
  if (n) n->err = msg;
  else g_mlp_err = msg;
  return s;
}

#define LB_MCUDA(n, call)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return mfail(n, LB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
cudaError_t alloc(lb_mlp* n, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
  if (e == cudaSuccess) {
    n->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

template <class TA, class TB>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const TA* A, long sam, long sak, const TB* B, long sbk,
                 long sbn, float* C, int ldc, int accumulate) {
  const dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  k_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, accumulate);
  return cudaGetLastError();
}

// Forward pass of n rows; the outputs (normalised) land in n->Yout.
cudaError_t forward(lb_mlp* net, const float* x, int n) {
  cudaStream_t s = net->stream;
  k_features<<<nblk(n), 256, 0, s>>>(x, n, net->np, net->nf, net->phi);
  const float* in = net->phi;
  for (int l = 0; l < net->depth; ++l) {
    const int fi = net->fan_in[l], fo = net->fan_out[l];
    const bool last = l == net->depth - 1;
    float* Zl = last ? net->Yout : net->Z[l];
    float* Hl = last ? net->Yout : net->H[l];
    // Z[i][o] = sum_k in[i][k] W[o][k]
    cudaError_t e = gemm(s, n, fo, fi, in, fi, 1, net->wb + net->w_off[l], 1, fi, Zl, fo, 0);
    if (e != cudaSuccess) return e;
    k_bias_act<<<nblk(size_t(n) * fo), 256, 0, s>>>(Zl, Hl, net->w + net->b_off[l], n, fo, last ? 0 : 1);
    in = Hl;
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

lb_status lb_mlp_create(int n_plain, int n_fourier, int width, int depth, int max_batch, unsigned long long seed,
                        void* cuda_stream, lb_mlp** out) {
  if (!out) return mfail(nullptr, LB_ERR_ARG, "null argument");
  *out = nullptr;
  if (n_plain < 1 || n_plain > 16 || n_fourier < 0 || n_fourier > 16 || width < 4 || width > 4096 || depth < 2 ||
      depth > 16 || max_batch < 1 || max_batch > (1 << 22))
    return mfail(nullptr, LB_ERR_ARG, "need 1 <= n_plain <= 16, 0 <= n_fourier <= 16, 4 <= width <= 4096, "
                                      "2 <= depth <= 16, 1 <= max_batch <= 4M");
  lb_mlp* n = new lb_mlp();
  n->np = n_plain;
  n->nf = n_fourier;
  n->width = width;
  n->depth = depth;
  n->max_batch = max_batch;
  n->nin = n_plain + 2 * n_fourier;
  n->stream = static_cast<cudaStream_t>(cuda_stream);
  for (int l = 0; l < depth; ++l) {
    n->fan_in.push_back(l == 0 ? n->nin : width);
    n->fan_out.push_back(l == depth - 1 ? NOUT : width);
  }
  for (int l = 0; l < depth; ++l) {
    n->w_off.push_back(n->nparam);
    n->nparam += size_t(n->fan_in[l]) * n->fan_out[l];
    n->b_off.push_back(n->nparam);
    n->nparam += size_t(n->fan_out[l]);
  }
  auto bail = [&](cudaError_t e) {
    const std::string m = std::string("allocation: ") + cudaGetErrorString(e);
    lb_mlp_destroy(n);
    return mfail(nullptr, LB_ERR_CUDA, m);
  };
  cudaError_t e = cudaSuccess;
  for (float** p : {&n->w, &n->g, &n->m, &n->v})
    if (e == cudaSuccess) e = alloc(n, p, n->nparam);
  if (e == cudaSuccess) e = alloc(n, &n->wb, n->nparam);
  if (e == cudaSuccess) e = alloc(n, &n->phi, size_t(max_batch) * n->nin);
  if (e == cudaSuccess) e = alloc(n, &n->Yout, size_t(max_batch) * NOUT);
  if (e == cudaSuccess) e = alloc(n, &n->dY, size_t(max_batch) * NOUT);
  if (e == cudaSuccess) e = alloc(n, &n->partial, nblk(size_t(max_batch) * NOUT) + 1);
  if (e == cudaSuccess) e = alloc(n, &n->loss, 1);
  if (e == cudaSuccess) e = alloc(n, &n->scale, 3 * NOUT);
  if (e == cudaSuccess) e = alloc(n, &n->dA, size_t(max_batch) * width);
  if (e == cudaSuccess) e = alloc(n, &n->dB, size_t(max_batch) * width);
  n->Z.assign(depth - 1, nullptr);
  n->H.assign(depth - 1, nullptr);
  for (int l = 0; l < depth - 1 && e == cudaSuccess; ++l) {
    e = alloc(n, &n->Z[l], size_t(max_batch) * width);
    if (e == cudaSuccess) e = alloc(n, &n->H[l], size_t(max_batch) * width);
  }
  if (e != cudaSuccess) return bail(e);
  // He-uniform initial weights (SplitMix64 stream), zero biases and moments
  std::vector<float> h(n->nparam, 0.0f);
  uint64_t k = 0;
  for (int l = 0; l < depth; ++l) {
    const double a = std::sqrt(6.0 / n->fan_in[l]) * (l == depth - 1 ? 0.5 : 1.0);
    for (size_t i = 0; i < size_t(n->fan_in[l]) * n->fan_out[l]; ++i) {
      uint64_t z = seed + (++k) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const double u = double(z >> 11) * 0x1.0p-53;
      h[n->w_off[l] + i] = float(a * (2.0 * u - 1.0));
    }
  }
  const float sc[3 * NOUT] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1};
  e = cudaMemcpy(n->w, h.data(), n->nparam * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, n->nparam * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, n->nparam * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(n->scale, sc, sizeof(sc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_to_bf16<<<nblk(n->nparam), 256, 0, n->stream>>>(n->w, n->wb, n->nparam);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return bail(e);
  *out = n;
  return LB_OK;
}

size_t lb_mlp_param_count(const lb_mlp* n) { return n ? n->nparam : 0; }

lb_status lb_mlp_set_output_scale(lb_mlp* n, const float* mean, const float* sd) {
  if (!n || !mean || !sd) return mfail(n, LB_ERR_ARG, "null argument");
  float h[3 * NOUT];
  for (int q = 0; q < NOUT; ++q) {
    if (!(sd[q] > 0.0f) || !std::isfinite(mean[q])) return mfail(n, LB_ERR_ARG, "need finite mean, std > 0");
    h[q] = mean[q];
    h[NOUT + q] = 1.0f / sd[q];
    h[2 * NOUT + q] = sd[q];
  }
  LB_MCUDA(n, cudaMemcpyAsync(n->scale, h, sizeof(h), cudaMemcpyHostToDevice, n->stream));
  LB_MCUDA(n, cudaStreamSynchronize(n->stream));
  return LB_OK;
}

lb_status lb_mlp_get_params(lb_mlp* n, float* host, size_t count) {
  if (!n || !host || count != n->nparam) return mfail(n, LB_ERR_ARG, "need a host buffer of lb_mlp_param_count floats");
  LB_MCUDA(n, cudaMemcpyAsync(host, n->w, count * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
  LB_MCUDA(n, cudaStreamSynchronize(n->stream));
  return LB_OK;
}

lb_status lb_mlp_set_params(lb_mlp* n, const float* host, size_t count) {
  if (!n || !host || count != n->nparam) return mfail(n, LB_ERR_ARG, "need a host buffer of lb_mlp_param_count floats");
  LB_MCUDA(n, cudaMemcpyAsync(n->w, host, count * sizeof(float), cudaMemcpyHostToDevice, n->stream));
  k_to_bf16<<<nblk(count), 256, 0, n->stream>>>(n->w, n->wb, count);
  LB_MCUDA(n, cudaGetLastError());
  LB_MCUDA(n, cudaMemsetAsync(n->m, 0, count * sizeof(float), n->stream));
  LB_MCUDA(n, cudaMemsetAsync(n->v, 0, count * sizeof(float), n->stream));
  LB_MCUDA(n, cudaStreamSynchronize(n->stream));
  n->steps = 0;
  return LB_OK;
}

lb_status lb_mlp_predict(lb_mlp* n, const float* x, int count, float* y) {
  if (!n || (!x && count) || (!y && count)) return mfail(n, LB_ERR_ARG, "null argument");
  if (count < 0 || count > n->max_batch) return mfail(n, LB_ERR_ARG, "need 0 <= count <= max_batch");
  if (count == 0) return LB_OK;
  LB_MCUDA(n, forward(n, x, count));
  k_denorm<<<nblk(size_t(count) * NOUT), 256, 0, n->stream>>>(n->Yout, n->scale, n->scale + 2 * NOUT, count, y);
  LB_MCUDA(n, cudaGetLastError());
  return LB_OK;
}

lb_status lb_mlp_train_step(lb_mlp* n, const float* x, const float* y, int count, float lr, float* loss) {
  if (!n || !x || !y) return mfail(n, LB_ERR_ARG, "null argument");
  if (count < 1 || count > n->max_batch) return mfail(n, LB_ERR_ARG, "need 1 <= count <= max_batch");
  if (!(lr > 0.0f) || !std::isfinite(lr)) return mfail(n, LB_ERR_ARG, "need lr > 0");
  cudaStream_t s = n->stream;
  LB_MCUDA(n, forward(n, x, count));
  const unsigned nb = nblk(size_t(count) * NOUT);
  k_mse<<<nb, 256, 0, s>>>(n->Yout, y, n->scale, n->scale + NOUT, count, n->dY, n->partial);
  k_sum<<<1, 256, 0, s>>>(n->partial, int(nb), float(count * NOUT), n->loss);
  LB_MCUDA(n, cudaGetLastError());
  // backward: dZ of the output layer is dY
  const float* dZ = n->dY;
  float* bufs[2] = {n->dA, n->dB};
  for (int l = n->depth - 1; l >= 0; --l) {
    const int fi = n->fan_in[l], fo = n->fan_out[l];
    const float* in = l == 0 ? n->phi : n->H[l - 1];
    // dW[o][k] = sum_i dZ[i][o] in[i][k];  db[o] = sum_i dZ[i][o]
    LB_MCUDA(n, gemm(s, fo, fi, count, dZ, 1, fo, in, fi, 1, n->g + n->w_off[l], fi, 0));
    k_colsum<<<nblk(fo), 256, 0, s>>>(dZ, count, fo, n->g + n->b_off[l]);
    LB_MCUDA(n, cudaGetLastError());
    if (l == 0) break;
    // dH[i][k] = sum_o dZ[i][o] W[o][k], then through the SiLU of layer l-1
    float* dH = bufs[l & 1];
    LB_MCUDA(n, gemm(s, count, fi, fo, dZ, fo, 1, n->wb + n->w_off[l], fi, 1, dH, fi, 0));
    k_silu_back<<<nblk(size_t(count) * fi), 256, 0, s>>>(n->Z[l - 1], dH, size_t(count) * fi);
    LB_MCUDA(n, cudaGetLastError());
    dZ = dH;
  }
  ++n->steps;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, float(n->steps)), c2 = 1.0f - std::pow(b2, float(n->steps));
  k_adam<<<nblk(n->nparam), 256, 0, s>>>(n->w, n->g, n->m, n->v, n->wb, n->nparam, lr, b1, b2, c1, c2, 1e-8f);
  LB_MCUDA(n, cudaGetLastError());
  if (loss) {
    LB_MCUDA(n, cudaMemcpyAsync(loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    LB_MCUDA(n, cudaStreamSynchronize(s));
  }
  return LB_OK;
}

lb_status lb_mlp_get_grads(lb_mlp* n, float* host, size_t count) {
  if (!n || !host || count != n->nparam) return mfail(n, LB_ERR_ARG, "need a host buffer of lb_mlp_param_count floats");
  LB_MCUDA(n, cudaMemcpyAsync(host, n->g, count * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
  LB_MCUDA(n, cudaStreamSynchronize(n->stream));
  return LB_OK;
}

void lb_mlp_destroy(lb_mlp* n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  else cudaDeviceSynchronize();
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

const char* lb_mlp_last_error(const lb_mlp* n) { return n ? n->err.c_str() : g_mlp_err.c_str(); }

}  // extern "C"
