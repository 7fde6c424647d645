// k_mlp.cu -- the learned tuner's network: forward, backward and Adam as
// hand-written FP32 kernels (no tensor cores: the whole network has ~7k
// parameters and batches of at most a few thousand rows).
//
// The paper proposes knowledge-based or data-driven tuning as future work
// (Sec. 6) to avoid full search's cost of executing every configuration in
// every tuning phase (Sec. 2.3.2).  Here a 16-64-64-C MLP (tanh, tanh,
// linear) maps the 16 features of a particle system to the predicted log
// force time of each configuration; training minimises the masked mean
// squared error over measured (features, configuration, log time) rows.
//
// Parameter layout: W1[64][16] b1[64] W2[64][64] b2[64] W3[C][64] b3[C].
// Weight gradients are reductions over the rows in a fixed order (no atomics),
// so training is deterministic.  One full-batch epoch (forward, backward,
// gradient reductions, Adam) is captured once as a CUDA graph and replayed.
#include <cmath>
#include <vector>

#include "ljgb_internal.cuh"

namespace ljgb {

constexpr int MIN_ = 16, MH = 64;

__host__ __device__ inline int64_t mlp_nparams(int C) { return MH * MIN_ + MH + MH * MH + MH + (int64_t)C * MH + C; }

struct MlpPtr {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};

__device__ __forceinline__ MlpPtr mlp_ptrs(const float* p, int C) {
  MlpPtr q;
  q.W1 = p;
  q.b1 = q.W1 + MH * MIN_;
  q.W2 = q.b1 + MH;
  q.b2 = q.W2 + MH * MH;
  q.W3 = q.b2 + MH;
  q.b3 = q.W3 + (int64_t)C * MH;
  return q;
}

// One block of 64 threads per row.
__global__ void __launch_bounds__(64) k_mlp_forward(const float* __restrict__ p, int C, const float* __restrict__ X,
                                                    int64_t M, float* __restrict__ H1, float* __restrict__ H2,
                                                    float* __restrict__ Y) {
  __shared__ float sx[MIN_], s1[MH], s2[MH];
  const int64_t m = blockIdx.x;
  const int h = threadIdx.x;
  if (m >= M) return;
  const MlpPtr q = mlp_ptrs(p, C);
  if (h < MIN_) sx[h] = X[m * MIN_ + h];
  __syncthreads();
  float a = q.b1[h];
#pragma unroll
  for (int i = 0; i < MIN_; ++i) a = fmaf(q.W1[h * MIN_ + i], sx[i], a);
  s1[h] = tanhf(a);
  if (H1) H1[m * MH + h] = s1[h];
  __syncthreads();
  a = q.b2[h];
#pragma unroll 8
  for (int i = 0; i < MH; ++i) a = fmaf(q.W2[h * MH + i], s1[i], a);
  s2[h] = tanhf(a);
  if (H2) H2[m * MH + h] = s2[h];
  __syncthreads();
  for (int c = h; c < C; c += MH) {
    float y = q.b3[c];
#pragma unroll 8
    for (int i = 0; i < MH; ++i) y = fmaf(q.W3[c * MH + i], s2[i], y);
    Y[m * C + c] = y;
  }
}

// Per-row backward: dY = 2 mask (y - t) / msum; D2 = (1 - h2^2) W3^T dY;
// D1 = (1 - h1^2) W2^T D2; row loss mask (y - t)^2.
__global__ void __launch_bounds__(64) k_mlp_backward_rows(const float* __restrict__ p, int C, int64_t M,
                                                          const float* __restrict__ T, const float* __restrict__ mask,
                                                          const float* __restrict__ msum, const float* __restrict__ H1,
                                                          const float* __restrict__ H2, const float* __restrict__ Y,
                                                          float* __restrict__ DY, float* __restrict__ D1,
                                                          float* __restrict__ D2, float* __restrict__ rowloss) {
  extern __shared__ float sdy[];  // C floats
  __shared__ float sd2[MH];
  __shared__ float sl[MH];
  const int64_t m = blockIdx.x;
  const int h = threadIdx.x;
  if (m >= M) return;
  const MlpPtr q = mlp_ptrs(p, C);
  const float inv = 1.0f / *msum;
  float l = 0.0f;
  for (int c = h; c < C; c += MH) {
    const float e = Y[m * C + c] - T[m * C + c];
    const float w = mask[m * C + c];
    sdy[c] = 2.0f * w * e * inv;
    DY[m * C + c] = sdy[c];
    l += w * e * e;
  }
  sl[h] = l;
  __syncthreads();
  float a = 0.0f;
  for (int c = 0; c < C; ++c) a = fmaf(q.W3[c * MH + h], sdy[c], a);
  const float h2 = H2[m * MH + h];
  sd2[h] = a * (1.0f - h2 * h2);
  D2[m * MH + h] = sd2[h];
  __syncthreads();
  a = 0.0f;
#pragma unroll 8
  for (int o = 0; o < MH; ++o) a = fmaf(q.W2[o * MH + h], sd2[o], a);
  const float h1 = H1[m * MH + h];
  D1[m * MH + h] = a * (1.0f - h1 * h1);
  if (h == 0) {
    float t = 0.0f;
    for (int k = 0; k < MH; ++k) t += sl[k];
    rowloss[m] = t;
  }
}

// gW[o][k] = sum_m D[m][o] A[m][k] (k < K), gb[o] = sum_m D[m][o] (the column
// k = K).  Block (o, 32-column chunk): lane tx takes column 32 chunk + tx,
// row group ty the rows m = ty, ty + WG_ROWS, ...; the WG_ROWS partial sums of
// a column are added in a fixed order in shared memory, so the result does not
// depend on scheduling.  The row loads of A are coalesced over the columns and
// D[m][o] is broadcast.
constexpr int WG_ROWS = 32;
__global__ void __launch_bounds__(32 * WG_ROWS) k_mlp_wgrad(const float* __restrict__ A, int K,
                                                           const float* __restrict__ D, int O, int64_t M,
                                                           float* __restrict__ gW, float* __restrict__ gb) {
  __shared__ float part[WG_ROWS][33];
  const int o = blockIdx.x, tx = threadIdx.x, ty = threadIdx.y;
  const int k = blockIdx.y * 32 + tx;
  float s = 0.0f;
  if (k <= K) {
#pragma unroll 4
    for (int64_t m = ty; m < M; m += WG_ROWS) {
      const float d = D[m * O + o];
      s = k < K ? fmaf(d, A[m * K + k], s) : s + d;
    }
  }
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && k <= K) {
    float t = 0.0f;
    for (int r = 0; r < WG_ROWS; ++r) t += part[r][tx];
    if (k < K) gW[o * K + k] = t;
    else gb[o] = t;
  }
}

__global__ void k_mlp_loss(const float* __restrict__ rowloss, int64_t M, const float* __restrict__ msum,
                           float* __restrict__ out, const int* __restrict__ step) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float s = 0.0f;
  for (int64_t m = 0; m < M; ++m) s += rowloss[m];
  out[step ? *step : 0] = s / *msum;
}

// Adam (Kingma & Ba 2015) with bias corrections from the device step counter.
__global__ void k_adam_prep(int* __restrict__ step, float* __restrict__ corr, float b1, float b2) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int t = ++(*step);
    corr[0] = 1.0f - powf(b1, (float)t);
    corr[1] = 1.0f - powf(b2, (float)t);
  }
}

__global__ void k_adam(int64_t P, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, const float* __restrict__ corr) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk;
  const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / corr[0]) / (sqrtf(vk / corr[1]) + eps);
}

// Training inputs of the learned tuner.  Row m of the timings (NaN or non-
// positive = not timed): Y = log(t / t_best) over the valid entries, 0 and a
// zero mask elsewhere; one warp per row, its lanes over the configurations
// (the row's best by a warp minimum).
__global__ void k_tuner_targets(const double* __restrict__ T, int64_t M, int C, float* __restrict__ Y,
                                float* __restrict__ mask) {
  const int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (m >= M) return;  // whole warps leave together
  double best = INFINITY;
  for (int c = lane; c < C; c += 32) {
    const double t = T[m * C + c];
    if (isfinite(t) && t > 0.0 && t < best) best = t;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  for (int c = lane; c < C; c += 32) {
    const double t = T[m * C + c];
    const bool ok = isfinite(t) && t > 0.0;
    Y[m * C + c] = ok ? (float)log(t / best) : 0.0f;
    mask[m * C + c] = ok ? 1.0f : 0.0f;
  }
}

// Mean and population standard deviation of feature f over the rows (block
// f; FP64 partial sums in a fixed tree order), a deviation below 1e-12
// replaced by 1; then the standardised features.
constexpr int STD_T = 256;
__global__ void __launch_bounds__(STD_T) k_feature_moments(const double* __restrict__ X, int64_t M, int F,
                                                           double* __restrict__ mom) {
  __shared__ double sh[STD_T];
  const int f = blockIdx.x, t = threadIdx.x;
  double s = 0.0;
  for (int64_t m = t; m < M; m += STD_T) s += X[m * F + f];
  sh[t] = s;
  __syncthreads();
  for (int o = STD_T / 2; o > 0; o >>= 1) {
    if (t < o) sh[t] += sh[t + o];
    __syncthreads();
  }
  const double mu = sh[0] / (double)M;
  __syncthreads();
  double q = 0.0;
  for (int64_t m = t; m < M; m += STD_T) q += (X[m * F + f] - mu) * (X[m * F + f] - mu);
  sh[t] = q;
  __syncthreads();
  for (int o = STD_T / 2; o > 0; o >>= 1) {
    if (t < o) sh[t] += sh[t + o];
    __syncthreads();
  }
  if (t == 0) {
    const double sd = sqrt(sh[0] / (double)M);
    mom[2 * f] = mu;
    mom[2 * f + 1] = sd < 1e-12 ? 1.0 : sd;
  }
}

__global__ void k_standardize(const double* __restrict__ X, int64_t M, int F, const double* __restrict__ mom,
                              float* __restrict__ Xs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * F) return;
  const int f = (int)(e % F);
  Xs[e] = (float)((X[e] - mom[2 * f]) / mom[2 * f + 1]);
}

// Device workspace for one (M, C) problem.
struct MlpWork {
  int64_t M = 0;
  int C = 0;
  float *p = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;
  float *X = nullptr, *T = nullptr, *mask = nullptr, *msum = nullptr;
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *DY = nullptr, *D1 = nullptr, *D2 = nullptr;
  float *rowloss = nullptr, *losses = nullptr, *corr = nullptr;
  int* step = nullptr;
  ~MlpWork() {
    float* fs[] = {p, g, am, av, X, T, mask, msum, H1, H2, Y, DY, D1, D2, rowloss, losses, corr};
    for (float* f : fs)
      if (f) cudaFree(f);
    if (step) cudaFree(step);
  }
};

static cudaError_t mlp_alloc(MlpWork& w, int64_t M, int C, int epochs) {
  const int64_t P = mlp_nparams(C);
  w.M = M;
  w.C = C;
  cudaError_t e = cudaSuccess;
  auto A = [&](float*& q, int64_t k) {
    if (e == cudaSuccess) e = cudaMalloc(&q, (size_t)std::max<int64_t>(k, 1) * sizeof(float));
  };
  A(w.p, P);
  A(w.g, P);
  A(w.am, P);
  A(w.av, P);
  A(w.X, M * MIN_);
  A(w.T, M * C);
  A(w.mask, M * C);
  A(w.msum, 1);
  A(w.H1, M * MH);
  A(w.H2, M * MH);
  A(w.Y, M * C);
  A(w.DY, M * C);
  A(w.D1, M * MH);
  A(w.D2, M * MH);
  A(w.rowloss, M);
  A(w.losses, epochs + 1);
  A(w.corr, 2);
  if (e == cudaSuccess) e = cudaMalloc(&w.step, sizeof(int));
  return e;
}

// Forward + backward + gradient reductions; grad in w.g, loss in w.losses[*step].
static cudaError_t mlp_fwd_bwd(MlpWork& w, cudaStream_t s) {
  const int C = w.C;
  const int64_t M = w.M;
  k_mlp_forward<<<(unsigned)M, MH, 0, s>>>(w.p, C, w.X, M, w.H1, w.H2, w.Y);
  k_mlp_backward_rows<<<(unsigned)M, MH, C * sizeof(float), s>>>(w.p, C, M, w.T, w.mask, w.msum, w.H1, w.H2, w.Y,
                                                                 w.DY, w.D1, w.D2, w.rowloss);
  float* gW1 = w.g;
  float* gb1 = gW1 + MH * MIN_;
  float* gW2 = gb1 + MH;
  float* gb2 = gW2 + MH * MH;
  float* gW3 = gb2 + MH;
  float* gb3 = gW3 + (int64_t)C * MH;
  const dim3 wb(32, WG_ROWS);
  k_mlp_wgrad<<<dim3(MH, (MIN_ + 32) / 32), wb, 0, s>>>(w.X, MIN_, w.D1, MH, M, gW1, gb1);
  k_mlp_wgrad<<<dim3(MH, (MH + 32) / 32), wb, 0, s>>>(w.H1, MH, w.D2, MH, M, gW2, gb2);
  k_mlp_wgrad<<<dim3(C, (MH + 32) / 32), wb, 0, s>>>(w.H2, MH, w.DY, C, M, gW3, gb3);
  k_mlp_loss<<<1, 32, 0, s>>>(w.rowloss, M, w.msum, w.losses, w.step);
  return cudaGetLastError();
}

static cudaError_t mlp_upload(MlpWork& w, const float* params, const float* X, const float* T, const float* mask,
                              cudaStream_t s) {
  const int64_t M = w.M, P = mlp_nparams(w.C);
  const int C = w.C;
  cudaError_t e = cudaMemcpyAsync(w.p, params, P * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.X, X, M * MIN_ * sizeof(float), cudaMemcpyHostToDevice, s);
  if (T && e == cudaSuccess) e = cudaMemcpyAsync(w.T, T, M * C * sizeof(float), cudaMemcpyHostToDevice, s);
  if (mask && e == cudaSuccess) {
    e = cudaMemcpyAsync(w.mask, mask, M * C * sizeof(float), cudaMemcpyHostToDevice, s);
    double ms = 0.0;
    for (int64_t k = 0; k < M * C; ++k) ms += mask[k];
    static thread_local float h_ms;
    h_ms = (float)(ms > 0 ? ms : 1.0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.msum, &h_ms, sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w.step, 0, sizeof(int), s);
  return e;
}

cudaError_t mlp_forward_dev(const float* d_params, int C, const float* d_X, int64_t M, float* d_Y, cudaStream_t s) {
  k_mlp_forward<<<(unsigned)M, MH, 0, s>>>(d_params, C, d_X, M, nullptr, nullptr, d_Y);
  return cudaGetLastError();
}

}  // namespace ljgb

using namespace ljgb;

extern "C" {

/* See include/ljgb.h. */
lj_status lj_mlp_forward(const float* params, int32_t C, const float* X, int64_t M, float* Y, void* stream) {
  if (!params || !X || !Y || C < 1 || M < 1) return LJ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  MlpWork w;
  if (mlp_alloc(w, M, C, 0) != cudaSuccess) return LJ_ERR_OOM;
  if (mlp_upload(w, params, X, nullptr, nullptr, s) != cudaSuccess) return LJ_ERR_CUDA;
  k_mlp_forward<<<(unsigned)M, MH, 0, s>>>(w.p, C, w.X, M, nullptr, nullptr, w.Y);
  if (cudaGetLastError() != cudaSuccess) return LJ_ERR_CUDA;
  if (cudaMemcpyAsync(Y, w.Y, M * C * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LJ_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? LJ_OK : LJ_ERR_CUDA;
}

lj_status lj_mlp_loss_grad(const float* params, int32_t C, const float* X, const float* T, const float* mask,
                           int64_t M, float* grad, float* loss, void* stream) {
  if (!params || !X || !T || !mask || !grad || C < 1 || M < 1) return LJ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  MlpWork w;
  if (mlp_alloc(w, M, C, 0) != cudaSuccess) return LJ_ERR_OOM;
  if (mlp_upload(w, params, X, T, mask, s) != cudaSuccess) return LJ_ERR_CUDA;
  if (mlp_fwd_bwd(w, s) != cudaSuccess) return LJ_ERR_CUDA;
  const int64_t P = mlp_nparams(C);
  if (cudaMemcpyAsync(grad, w.g, P * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LJ_ERR_CUDA;
  float l = 0.0f;
  if (cudaMemcpyAsync(&l, w.losses, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LJ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LJ_ERR_CUDA;
  if (loss) *loss = l;
  return LJ_OK;
}

lj_status lj_tuner_prepare(const double* T, int64_t M, int32_t C, const double* X, float* Y, float* mask, float* Xs,
                           float* mean, float* sd, void* stream) {
  if (!T || !X || !Y || !mask || !Xs || !mean || !sd || C < 1 || M < 1) return LJ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  double *dT = nullptr, *dX = nullptr, *dmom = nullptr;
  float *dY = nullptr, *dM = nullptr, *dXs = nullptr;
  const size_t nT = (size_t)M * C, nX = (size_t)M * MIN_;
  lj_status st = LJ_OK;
  if (cudaMalloc(&dT, nT * sizeof(double)) != cudaSuccess || cudaMalloc(&dX, nX * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dmom, 2 * MIN_ * sizeof(double)) != cudaSuccess || cudaMalloc(&dY, nT * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dM, nT * sizeof(float)) != cudaSuccess || cudaMalloc(&dXs, nX * sizeof(float)) != cudaSuccess)
    st = LJ_ERR_OOM;
  std::vector<double> mom(2 * MIN_);
  if (st == LJ_OK) {
    cudaError_t e = cudaMemcpyAsync(dT, T, nT * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dX, X, nX * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      k_tuner_targets<<<(unsigned)((M + 3) / 4), 128, 0, s>>>(dT, M, C, dY, dM);
      k_feature_moments<<<MIN_, STD_T, 0, s>>>(dX, M, MIN_, dmom);
      k_standardize<<<(unsigned)(((int64_t)nX + 255) / 256), 256, 0, s>>>(dX, M, MIN_, dmom, dXs);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(Y, dY, nT * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mask, dM, nT * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Xs, dXs, nX * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mom.data(), dmom, 2 * MIN_ * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = LJ_ERR_CUDA;
  }
  if (st == LJ_OK)
    for (int f = 0; f < MIN_; ++f) {
      mean[f] = (float)mom[2 * f];
      sd[f] = (float)mom[2 * f + 1];
    }
  for (void* p : {(void*)dT, (void*)dX, (void*)dmom, (void*)dY, (void*)dM, (void*)dXs})
    if (p) cudaFree(p);
  return st;
}

lj_status lj_mlp_train(const float* X, const float* T, const float* mask, int64_t M, int32_t C, float* params,
                       int32_t epochs, float lr, float* losses, void* stream) {
  if (!X || !T || !mask || !params || C < 1 || M < 1 || epochs < 0 || !(lr > 0)) return LJ_ERR_ARG;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LJ_ERR_CUDA;
  (void)stream;
  lj_status st = LJ_OK;
  {
    MlpWork w;
    const int64_t P = mlp_nparams(C);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (mlp_alloc(w, M, C, epochs) != cudaSuccess) st = LJ_ERR_OOM;
    if (st == LJ_OK && mlp_upload(w, params, X, T, mask, s) != cudaSuccess) st = LJ_ERR_CUDA;
    if (st == LJ_OK && (cudaMemsetAsync(w.am, 0, P * sizeof(float), s) != cudaSuccess ||
                        cudaMemsetAsync(w.av, 0, P * sizeof(float), s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
      st = LJ_ERR_CUDA;
    if (st == LJ_OK) {
      // one epoch: loss/gradients at the current parameters (loss stored at
      // index step), then the step counter and the Adam update
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) e = mlp_fwd_bwd(w, s);
      if (e == cudaSuccess) {
        k_adam_prep<<<1, 32, 0, s>>>(w.step, w.corr, 0.9f, 0.999f);
        k_adam<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(P, w.p, w.g, w.am, w.av, lr, 0.9f, 0.999f, 1e-8f, w.corr);
        e = cudaGetLastError();
      }
      cudaError_t e2 = cudaStreamEndCapture(s, &graph);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      for (int32_t k = 0; e == cudaSuccess && k < epochs; ++k) e = cudaGraphLaunch(exec, s);
      // final loss at the trained parameters
      if (e == cudaSuccess) e = mlp_fwd_bwd(w, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(params, w.p, P * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (losses && e == cudaSuccess)
        e = cudaMemcpyAsync(losses, w.losses, (size_t)(epochs + 1) * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = LJ_ERR_CUDA;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  cudaStreamDestroy(s);
  return st;
}

}  // extern "C"
