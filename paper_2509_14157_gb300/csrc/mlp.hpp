// Per-amplitude MLP of the learned Davidson guess (training and inference
// on the device). See mlp.cu.
#pragma once
#include "common.hpp"

#include <cstdint>
#include <memory>
#include <string>

namespace fnocc {

constexpr int kMlpFeatures = 8;  // per-amplitude features (see eom_features)
constexpr int kMlpOutputs = 2;   // guess importance, diagonal correction

// features [nhtup * nptup x kMlpFeatures] of one packed EOM component
// (n active spin orbitals, g their antisymmetrised integrals)
void eom_features(cudaStream_t s, int nh, int np, int o, int n, const int *htab, long long nhtup, const int *ptab,
                  long long nptup, const double *fdiag, const double *g, const float *vocc_log, int comp, int variant,
                  float *out);

// dg[i] += clamp(y[i * stride + col], -clamp, clamp)
void add_diag_correction(cudaStream_t s, long long n, const float *y, int stride, int col, double clamp, double *dg);

class Mlp {
 public:
  Mlp(int device, int nin, int width, int nout, uint64_t seed);
  ~Mlp();
  Mlp(const Mlp &) = delete;
  Mlp &operator=(const Mlp &) = delete;
  size_t nparam() const { return nparam_; }
  int nin() const { return nin_; }
  int width() const { return width_; }
  int nout() const { return nout_; }
  int device() const { return device_; }
  // parameters: W1 [nin x width], b1, W2 [width x width], b2, W3 [width x nout], b3
  // (row-major, input index first), FP32
  void set_params(const float *host);
  void get_params(float *host) const;
  void reset_optimizer();
  // loss = sum_i sum_o Wt[i,o] (Y[i,o] - T[i,o])^2 / n over n device rows;
  // gradient into the internal gradient buffer (same layout as the parameters)
  double loss_grad(const float *X, const float *T, const float *Wt, int n);
  const float *grad() const { return grad_.as<float>(); }
  void adam_step(float lr, float b1, float b2, float eps);
  // minibatch Adam over host data; history[epoch] = mean training loss
  void train(const float *X, const float *T, const float *Wt, long long n, int epochs, int batch, float lr,
             uint64_t seed, double *history);
  // parameters are only read: concurrent calls on different streams are safe
  // when each passes its own scratch
  void infer_bf16(const float *X, long long n, float *Y, cudaStream_t stream, DevBuf &scratch) const;
  void infer_fp32(const float *X, long long n, float *Y);
  cudaStream_t stream() const { return stream_; }

 private:
  void forward_train(const float *X, int n);
  const float *W(int l) const;
  const float *b(int l) const;
  int device_, nin_, width_, nout_;
  size_t nparam_ = 0, woff_[3] = {0, 0, 0}, boff_[3] = {0, 0, 0};
  cudaStream_t stream_ = nullptr;
  DevBuf params_, grad_, adam_m_, adam_v_, act_, dact_, part_, lossp_, ones_, data_, mb_, rows_;
  int adam_t_ = 0;
};

}  // namespace fnocc

// C-ABI handle (include/fnocc.h)
struct fnocc_mlp {
  std::unique_ptr<fnocc::Mlp> net;
  std::string err;
};
