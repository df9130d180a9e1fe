// mlp.cu -- a8: the cost model's network, trained and evaluated on the GPU.
//
// The planner predicts the log run time of a closure configuration from a feature vector x
// (log n, edge density, dtype, algorithm, cutoff) with a two-hidden-layer perceptron:
//     h1 = relu(x W1 + b1),  h2 = relu(h1 W2 + b2),  y = h2 . w3 + b3,
// width 64, fp32.  These kernels are its forward pass, the mean-squared-error loss and its
// gradient, the backward pass (deterministic: per-block partial gradients, then a fixed-order
// reduction) and an Adam update.  They are small: throughput is irrelevant next to a closure.
//
// Parameter layout (one flat float array): W1 [in x 64] row-major, b1 [64], W2 [64 x 64]
// row-major, b2 [64], w3 [64], b3 [1].
#include "common.cuh"

namespace apsp {

constexpr int kH = 64;          // hidden width
constexpr int kMlpMaxIn = 32;   // largest feature dimension
constexpr int kSamplesPerBlock = 32;

__host__ __device__ inline int64_t mlp_param_count(int in) { return (int64_t)in * kH + kH + kH * kH + kH + kH + 1; }

struct MlpParams {
  const float *W1, *b1, *W2, *b2, *w3, *b3;
};
__device__ __forceinline__ MlpParams split_params(const float *p, int in) {
  MlpParams m;
  m.W1 = p;
  m.b1 = m.W1 + in * kH;
  m.W2 = m.b1 + kH;
  m.b2 = m.W2 + kH * kH;
  m.w3 = m.b2 + kH;
  m.b3 = m.w3 + kH;
  return m;
}

// One block: 64 threads (one per hidden unit) x up to 32 samples.  acts (optional) receives
// h1 and h2 per sample: [batch][2][64].
__global__ void __launch_bounds__(kH) mlp_forward_kernel(const float *params, int in, const float *x, int batch,
                                                         float *out, float *acts) {
  __shared__ float xs[kSamplesPerBlock][kMlpMaxIn];
  __shared__ float h1s[kSamplesPerBlock][kH];
  __shared__ float part[kSamplesPerBlock][kH];
  const MlpParams P = split_params(params, in);
  const int j = threadIdx.x;
  const int s0 = blockIdx.x * kSamplesPerBlock;
  const int ns = min(kSamplesPerBlock, batch - s0);
  for (int e = j; e < ns * in; e += kH) xs[e / in][e % in] = x[(int64_t)(s0 + e / in) * in + e % in];
  __syncthreads();
  for (int s = 0; s < ns; ++s) {
    float z = P.b1[j];
    for (int i = 0; i < in; ++i) z = fmaf(xs[s][i], P.W1[i * kH + j], z);
    h1s[s][j] = fmaxf(z, 0.0f);
  }
  __syncthreads();
  for (int s = 0; s < ns; ++s) {
    float z = P.b2[j];
    for (int k = 0; k < kH; ++k) z = fmaf(h1s[s][k], P.W2[k * kH + j], z);
    const float h2 = fmaxf(z, 0.0f);
    part[s][j] = h2 * P.w3[j];
    if (acts) {
      acts[(int64_t)(s0 + s) * 2 * kH + j] = h1s[s][j];
      acts[(int64_t)(s0 + s) * 2 * kH + kH + j] = h2;
    }
  }
  __syncthreads();
  if (j < ns) {  // fixed-order sum over the hidden units
    float y = P.b3[0];
    for (int k = 0; k < kH; ++k) y += part[j][k];
    out[s0 + j] = y;
  }
}

// Mean squared error L = mean((out - y)^2) and dL/dout = 2 (out - y) / batch (one block).
__global__ void __launch_bounds__(256) mlp_loss_kernel(const float *out, const float *y, int batch, float *dout,
                                                       float *loss) {
  __shared__ float red[256];
  float acc = 0.0f;
  for (int s = threadIdx.x; s < batch; s += blockDim.x) {
    const float e = out[s] - y[s];
    dout[s] = 2.0f * e / (float)batch;
    acc += e * e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = red[0] / (float)batch;
}

// Backward pass of one block of samples into its own slice of `partial` (one gradient-sized
// slice per block); mlp_reduce_kernel then sums the slices in block order.
__global__ void __launch_bounds__(kH) mlp_backward_kernel(const float *params, int in, const float *x,
                                                          const float *acts, const float *dout, int batch,
                                                          float *partial) {
  __shared__ float xs[kSamplesPerBlock][kMlpMaxIn];
  __shared__ float h1s[kSamplesPerBlock][kH];
  __shared__ float dz2s[kSamplesPerBlock][kH];
  __shared__ float dz1s[kSamplesPerBlock][kH];
  const MlpParams P = split_params(params, in);
  const int64_t np = mlp_param_count(in);
  float *g = partial + (int64_t)blockIdx.x * np;
  float *gW1 = g, *gb1 = gW1 + in * kH, *gW2 = gb1 + kH, *gb2 = gW2 + kH * kH, *gw3 = gb2 + kH, *gb3 = gw3 + kH;
  const int j = threadIdx.x;
  const int s0 = blockIdx.x * kSamplesPerBlock;
  const int ns = min(kSamplesPerBlock, batch - s0);
  for (int e = j; e < ns * in; e += kH) xs[e / in][e % in] = x[(int64_t)(s0 + e / in) * in + e % in];
  float gw3j = 0.0f, gb2j = 0.0f;
  for (int s = 0; s < ns; ++s) {
    const float *a = acts + (int64_t)(s0 + s) * 2 * kH;
    h1s[s][j] = a[j];
    const float h2 = a[kH + j];
    const float d = dout[s0 + s];
    gw3j += h2 * d;
    const float dz2 = h2 > 0.0f ? P.w3[j] * d : 0.0f;
    dz2s[s][j] = dz2;
    gb2j += dz2;
  }
  gw3[j] = gw3j;
  gb2[j] = gb2j;
  if (j == 0) {
    float t = 0.0f;
    for (int s = 0; s < ns; ++s) t += dout[s0 + s];
    gb3[0] = t;
  }
  __syncthreads();
  // dW2[k][j] = sum_s h1[s][k] dz2[s][j]; thread j owns column j
  for (int k = 0; k < kH; ++k) {
    float t = 0.0f;
    for (int s = 0; s < ns; ++s) t = fmaf(h1s[s][k], dz2s[s][j], t);
    gW2[k * kH + j] = t;
  }
  // dz1[s][k] (thread j plays k) = (h1 > 0) * sum_c W2[k][c] dz2[s][c]
  for (int s = 0; s < ns; ++s) {
    float t = 0.0f;
    for (int c = 0; c < kH; ++c) t = fmaf(P.W2[j * kH + c], dz2s[s][c], t);
    dz1s[s][j] = h1s[s][j] > 0.0f ? t : 0.0f;
  }
  __syncthreads();
  float gb1j = 0.0f;
  for (int s = 0; s < ns; ++s) gb1j += dz1s[s][j];
  gb1[j] = gb1j;
  for (int i = 0; i < in; ++i) {
    float t = 0.0f;
    for (int s = 0; s < ns; ++s) t = fmaf(xs[s][i], dz1s[s][j], t);
    gW1[i * kH + j] = t;
  }
}

__global__ void mlp_reduce_kernel(const float *partial, int nblocks, int64_t np, float *grads) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.x * blockDim.x) {
    float t = 0.0f;
    for (int b = 0; b < nblocks; ++b) t += partial[(int64_t)b * np + e];
    grads[e] = t;
  }
}

// Adam: m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2; p -= lr mhat / (sqrt(vhat) + eps).
__global__ void mlp_adam_kernel(float *p, const float *g, float *m, float *v, int64_t count, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace apsp

using namespace apsp;

extern "C" int64_t apsp_mlp_param_count(int in_dim) { return in_dim >= 1 && in_dim <= kMlpMaxIn ? mlp_param_count(in_dim) : -1; }

extern "C" size_t apsp_mlp_backward_workspace_bytes(int in_dim, int batch) {
  if (in_dim < 1 || in_dim > kMlpMaxIn || batch < 0) return 0;
  return (size_t)((batch + kSamplesPerBlock - 1) / kSamplesPerBlock) * (size_t)mlp_param_count(in_dim) * 4;
}

extern "C" int apsp_mlp_forward(const float *params, int in_dim, const float *x, int batch, float *out, float *acts,
                                void *stream) {
  if (in_dim < 1 || in_dim > kMlpMaxIn || batch < 0 || (batch > 0 && (!params || !x || !out))) return APSP_ERR_ARG;
  if (batch == 0) return APSP_OK;
  const int blocks = (batch + kSamplesPerBlock - 1) / kSamplesPerBlock;
  mlp_forward_kernel<<<blocks, kH, 0, reinterpret_cast<cudaStream_t>(stream)>>>(params, in_dim, x, batch, out, acts);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

extern "C" int apsp_mlp_loss(const float *out, const float *y, int batch, float *dout, float *loss, void *stream) {
  if (batch <= 0 || !out || !y || !dout) return APSP_ERR_ARG;
  mlp_loss_kernel<<<1, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, y, batch, dout, loss);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

extern "C" int apsp_mlp_backward(const float *params, int in_dim, const float *x, const float *acts,
                                 const float *dout, int batch, float *grads, void *ws, size_t ws_bytes,
                                 void *stream) {
  if (in_dim < 1 || in_dim > kMlpMaxIn || batch <= 0 || !params || !x || !acts || !dout || !grads || !ws)
    return APSP_ERR_ARG;
  if (ws_bytes < apsp_mlp_backward_workspace_bytes(in_dim, batch)) return APSP_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = (batch + kSamplesPerBlock - 1) / kSamplesPerBlock;
  float *partial = reinterpret_cast<float *>(ws);
  mlp_backward_kernel<<<blocks, kH, 0, s>>>(params, in_dim, x, acts, dout, batch, partial);
  APSP_LAUNCH_CHECK();
  const int64_t np = mlp_param_count(in_dim);
  mlp_reduce_kernel<<<(int)((np + 255) / 256), 256, 0, s>>>(partial, blocks, np, grads);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}

extern "C" int apsp_mlp_adam(float *params, const float *grads, float *m, float *v, int64_t count, float lr,
                             float beta1, float beta2, float eps, int step, void *stream) {
  if (count <= 0 || !params || !grads || !m || !v || step < 1) return APSP_ERR_ARG;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  const int blocks = (int)((count + 255) / 256);
  mlp_adam_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      params, grads, m, v, count, lr, beta1, beta2, eps, c1, c2);
  APSP_LAUNCH_CHECK();
  return APSP_OK;
}
