// Warm-start network: x (din) -> GELU(W1 x + b1) (dh) -> W2 h + b2 (dout).
#pragma once

#include "common.cuh"

namespace katz {

struct Mlp {
  int din = 0, dh = 0, dout = 0;
  bool ready = false;
  int step_count = 0;
  // FP32 master parameters and gradients, layout W1 (dh x din), b1 (dh),
  // W2 (dout x dh), b2 (dout); Adam moments; BF16 weight copies used by the
  // forward and backward kernels
  DBuf<float> params, grads, mom, var;
  DBuf<__nv_bfloat16> w1b, w2b;

  float* W1() const { return params.p; }
  float* b1() const { return params.p + int64_t(dh) * din; }
  float* W2() const { return b1() + dh; }
  float* b2() const { return W2() + int64_t(dout) * dh; }
  float* gW1() const { return grads.p; }
  float* gb1() const { return grads.p + int64_t(dh) * din; }
  float* gW2() const { return gb1() + dh; }
  float* gb2() const { return gW2() + int64_t(dout) * dh; }
  int64_t n_params() const { return int64_t(dh) * din + dh + int64_t(dout) * dh + dout; }

  void init(int din, int dh, int dout, uint64_t seed, cudaStream_t s);
  void set_params(const float* host, cudaStream_t s);
  void refresh_bf16(cudaStream_t s);
  // Hp = W1 x + b1, H = GELU(Hp), Y = W2 H + b2 for m rows of X (m x din)
  void forward(const float* X, int m, float* Hp, float* H, float* Y, cudaStream_t s) const;
  // mean squared error against T (m x dout) and its gradients into grads;
  // returns the loss
  double loss_grad(const float* X, const float* T, int m, Workspace& ws, cudaStream_t s);
  void adamw(float lr, float wd, cudaStream_t s);
};

}  // namespace katz
