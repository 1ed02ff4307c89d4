// Two-layer warm-start network y = W2 GELU(W1 x + b1) + b2 (exact erf GELU)
// with BF16 weights, FP32 activations and FP32 accumulation; mean squared
// error loss, its gradients, and AdamW on FP32 master weights.
//
// Sizes are small (input 32, hidden 256, output r <= 128, batch <= 8192),
// so each layer is one thread per output element with the weight row read
// from shared memory.
#include <cmath>

#include "mlp.h"

namespace katz {

namespace {

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// out[i][o] = sum_k in[i][k] * W[o][k] + bias[o]  (W BF16, o < dout)
// optional: pre (same as out) receives the pre-activation; out = GELU(pre)
__global__ void dense_fwd_kernel(const float* __restrict__ in, int m, int din,
                                 const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                                 int dout, float* __restrict__ pre, float* __restrict__ out,
                                 int act) {
  extern __shared__ float wrow[];  // din floats of one output unit
  const int o = blockIdx.y;
  for (int k = threadIdx.x; k < din; k += blockDim.x) wrow[k] = __bfloat162float(W[int64_t(o) * din + k]);
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const float* x = in + int64_t(i) * din;
    float acc = bias[o];
    for (int k = 0; k < din; ++k) acc += x[k] * wrow[k];
    if (pre) pre[int64_t(i) * dout + o] = acc;
    out[int64_t(i) * dout + o] = act ? gelu(acc) : acc;
  }
}

// dY = (Y - T) / m ; loss += 0.5 * sum (Y - T)^2 / m
__global__ void mse_kernel(const float* Y, const float* T, int64_t total, float inv_m, float* dY,
                           double* loss) {
  double local = 0;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const float d = Y[e] - T[e];
    dY[e] = d * inv_m;
    local += 0.5 * double(d) * double(d) * double(inv_m);
  }
  local = warp_sum(local);
  if ((threadIdx.x & 31) == 0 && local != 0.0) atomicAdd(loss, local);
}

// dW[o][k] = sum_i dOut[i][o] * in[i][k] ; db[o] = sum_i dOut[i][o]
__global__ void dense_wgrad_kernel(const float* __restrict__ dOut, const float* __restrict__ in,
                                   int m, int din, int dout, float* __restrict__ dW,
                                   float* __restrict__ db) {
  const int o = blockIdx.x;
  for (int k = threadIdx.x; k <= din; k += blockDim.x) {
    float acc = 0.f;
    if (k < din) {
      for (int i = 0; i < m; ++i) acc += dOut[int64_t(i) * dout + o] * in[int64_t(i) * din + k];
      dW[int64_t(o) * din + k] = acc;
    } else {
      for (int i = 0; i < m; ++i) acc += dOut[int64_t(i) * dout + o];
      db[o] = acc;
    }
  }
}

// dIn[i][k] = (sum_o dOut[i][o] * W[o][k]) * GELU'(pre[i][k])
__global__ void dense_dgrad_kernel(const float* __restrict__ dOut, int m, int dout,
                                   const __nv_bfloat16* __restrict__ W, int din,
                                   const float* __restrict__ pre, float* __restrict__ dIn) {
  const int64_t total = int64_t(m) * din;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / din;
    const int k = int(e - i * din);
    float acc = 0.f;
    for (int o = 0; o < dout; ++o)
      acc += dOut[i * dout + o] * __bfloat162float(W[int64_t(o) * din + k]);
    dIn[e] = acc * gelu_grad(pre[e]);
  }
}

__global__ void adamw_kernel(float* p, const float* g, float* mom, float* var, int64_t n, float lr,
                             float b1, float b2, float eps, float wd, float c1, float c2,
                             __nv_bfloat16* pb) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * mom[e] + (1.f - b1) * gg;
    const float vv = b2 * var[e] + (1.f - b2) * gg * gg;
    mom[e] = mm;
    var[e] = vv;
    const float mh = mm / c1, vh = vv / c2;
    const float np = p[e] - lr * (mh / (sqrtf(vh) + eps) + wd * p[e]);
    p[e] = np;
    if (pb) pb[e] = __float2bfloat16(np);
  }
}

__global__ void to_bf16_kernel(const float* x, __nv_bfloat16* y, int64_t n) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    y[e] = __float2bfloat16(x[e]);
}

unsigned blocks(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 4096));
}

}  // namespace

void Mlp::init(int din_, int dh_, int dout_, uint64_t seed, cudaStream_t s) {
  din = din_;
  dh = dh_;
  dout = dout_;
  const int64_t n1 = int64_t(dh) * din, n2 = int64_t(dout) * dh;
  std::vector<float> h(n1 + dh + n2 + dout, 0.f);
  // deterministic uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64
  uint64_t st = seed;
  auto uni = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return float(double(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  };
  for (int64_t e = 0; e < n1; ++e) h[e] = uni() / std::sqrt(float(din));
  for (int64_t e = 0; e < n2; ++e) h[n1 + dh + e] = uni() / std::sqrt(float(dh));
  set_params(h.data(), s);
}

void Mlp::set_params(const float* host, cudaStream_t s) {
  const int64_t n1 = int64_t(dh) * din, n2 = int64_t(dout) * dh;
  const int64_t tot = n1 + dh + n2 + dout;
  params.alloc(tot);
  grads.alloc(tot);
  mom.alloc(tot);
  var.alloc(tot);
  w1b.alloc(n1);
  w2b.alloc(n2);
  KATZ_CUDA(cudaMemcpyAsync(params.p, host, 4 * tot, cudaMemcpyHostToDevice, s));
  KATZ_CUDA(cudaMemsetAsync(mom.p, 0, 4 * tot, s));
  KATZ_CUDA(cudaMemsetAsync(var.p, 0, 4 * tot, s));
  refresh_bf16(s);
  step_count = 0;
  ready = true;
}

void Mlp::refresh_bf16(cudaStream_t s) {
  const int64_t n1 = int64_t(dh) * din, n2 = int64_t(dout) * dh;
  to_bf16_kernel<<<blocks(n1), 256, 0, s>>>(W1(), w1b.p, n1);
  KATZ_CHECK_LAUNCH();
  to_bf16_kernel<<<blocks(n2), 256, 0, s>>>(W2(), w2b.p, n2);
  KATZ_CHECK_LAUNCH();
}

void Mlp::forward(const float* X, int m, float* Hp, float* H, float* Y, cudaStream_t s) const {
  dim3 g1((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, 128), 64)), dh);
  dense_fwd_kernel<<<g1, 128, din * sizeof(float), s>>>(X, m, din, w1b.p, b1(), dh, Hp, H, 1);
  KATZ_CHECK_LAUNCH();
  dim3 g2((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, 128), 64)), dout);
  dense_fwd_kernel<<<g2, 128, dh * sizeof(float), s>>>(H, m, dh, w2b.p, b2(), dout, nullptr, Y, 0);
  KATZ_CHECK_LAUNCH();
}

double Mlp::loss_grad(const float* X, const float* T, int m, Workspace& ws, cudaStream_t s) {
  float* Hp = ws.get<float>("mlp.Hp", size_t(m) * dh);
  float* H = ws.get<float>("mlp.H", size_t(m) * dh);
  float* Y = ws.get<float>("mlp.Y", size_t(m) * dout);
  float* dY = ws.get<float>("mlp.dY", size_t(m) * dout);
  float* dHp = ws.get<float>("mlp.dHp", size_t(m) * dh);
  double* loss = ws.get<double>("mlp.loss", 1);
  forward(X, m, Hp, H, Y, s);
  KATZ_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
  mse_kernel<<<blocks(int64_t(m) * dout), 256, 0, s>>>(Y, T, int64_t(m) * dout, 1.f / m, dY, loss);
  KATZ_CHECK_LAUNCH();
  dense_wgrad_kernel<<<dout, 256, 0, s>>>(dY, H, m, dh, dout, gW2(), gb2());
  KATZ_CHECK_LAUNCH();
  dense_dgrad_kernel<<<blocks(int64_t(m) * dh), 256, 0, s>>>(dY, m, dout, w2b.p, dh, Hp, dHp);
  KATZ_CHECK_LAUNCH();
  dense_wgrad_kernel<<<dh, 64, 0, s>>>(dHp, X, m, din, dh, gW1(), gb1());
  KATZ_CHECK_LAUNCH();
  double h = 0;
  KATZ_CUDA(cudaMemcpyAsync(&h, loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  KATZ_CUDA(cudaStreamSynchronize(s));
  return h;
}

void Mlp::adamw(float lr, float wd, cudaStream_t s) {
  ++step_count;
  const float b1c = 0.9f, b2c = 0.999f;
  const float c1 = 1.f - std::pow(b1c, float(step_count));
  const float c2 = 1.f - std::pow(b2c, float(step_count));
  const int64_t tot = int64_t(dh) * din + dh + int64_t(dout) * dh + dout;
  adamw_kernel<<<blocks(tot), 256, 0, s>>>(params.p, grads.p, mom.p, var.p, tot, lr, b1c, b2c,
                                           1e-8f, wd, c1, c2, nullptr);
  KATZ_CHECK_LAUNCH();
  refresh_bf16(s);
}

}  // namespace katz
