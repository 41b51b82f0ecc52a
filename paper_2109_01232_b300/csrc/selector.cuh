// selector.cuh -- the learned parameter selector: matrix features and a 16-64-64-32 MLP
// (inference, loss gradient, Adam training), all as plain CUDA kernels in FP32 with
// fixed-order sums (bitwise reproducible).  Included at the end of solver.cu.
//
// The selector maps 16 cheap features of A to one of 32 classes (restart length m in
// {25, 50, 100, 200} x polynomial degree in {0, 10, 25, 40} x inner storage FP32/FP16),
// each class carrying the inner tolerance chosen for it when the model was trained.  It is
// trained on the solver's own sweep timings (paper_2109_01232_b300/selector.py) and falls
// back to the fixed default (m 50, no polynomial, FP32, inner tolerance 1e-4) when it has no
// model or is not confident.  The network is tiny (7,328 weights), so these kernels are
// simple thread-per-output loops: there is no dense contraction worth tensor cores here.
#pragma once

namespace gm {

constexpr int SEL_NF = GMRES_SEL_FEATURES;
constexpr int SEL_NH = 64;
constexpr int SEL_NC = GMRES_SEL_CLASSES;
constexpr int SEL_NP = GMRES_SEL_PARAMS;
constexpr int FEAT_NT = 256;
constexpr int FEAT_STATS = 16;
// statistics: sums 0..8, maxima 9..13, minima 14..15
enum {
  FS_RATIO = 0, FS_FRO2, FS_DABS, FS_RELOFF, FS_RELOFF_N, FS_DIST, FS_NUM, FS_DEN, FS_DOM,
  FS_MAXLEN, FS_INF, FS_AMAX, FS_DMAX, FS_DISTMAX, FS_RATIO_MIN, FS_DMIN_NZ
};

__device__ __forceinline__ double fs_combine(int k, double a, double b) {
  if (k <= FS_DOM) return a + b;
  if (k <= FS_DISTMAX) return fmax(a, b);
  return fmin(a, b);
}
__device__ __forceinline__ double fs_identity(int k) {
  return k <= FS_DOM ? 0.0 : (k <= FS_DISTMAX ? 0.0 : INFINITY);
}

// Per-CTA statistics of the rows (thread per row, grid-stride), combined in fixed order.
__global__ void __launch_bounds__(FEAT_NT) k_features_partial(const int* __restrict__ rp,
                                                              const int* __restrict__ ci,
                                                              const double* __restrict__ av, int n,
                                                              double* __restrict__ part) {
  double st[FEAT_STATS];
#pragma unroll
  for (int k = 0; k < FEAT_STATS; ++k) st[k] = fs_identity(k);
  for (long long i = blockIdx.x * (long long)FEAT_NT + threadIdx.x; i < n;
       i += (long long)gridDim.x * FEAT_NT) {
    const int k0 = rp[i], k1 = rp[i + 1];
    double s = 0.0, d = 0.0, so = 0.0;
    for (int k = k0; k < k1; ++k) {
      const int j = ci[k];
      const double a = av[k];
      s += fabs(a);
      st[FS_FRO2] += a * a;
      st[FS_AMAX] = fmax(st[FS_AMAX], fabs(a));
      const double dist = fabs((double)(i - j));
      st[FS_DIST] += dist;
      st[FS_DISTMAX] = fmax(st[FS_DISTMAX], dist);
      if (j == i) {
        d += a;
      } else {
        so += a;
        double aji = 0.0;  // the transposed entry (0 if row j does not hold column i)
        for (int kk = rp[j]; kk < rp[j + 1]; ++kk)
          if (ci[kk] == i) aji += av[kk];
        st[FS_NUM] += (a - aji) * (a - aji);
        st[FS_DEN] += a * a + aji * aji;
      }
    }
    const double ad = fabs(d);
    const double ratio = s > 0.0 ? ad / s : 0.0;
    st[FS_RATIO] += ratio;
    st[FS_RATIO_MIN] = fmin(st[FS_RATIO_MIN], ratio);
    st[FS_DABS] += ad;
    st[FS_DOM] += ad >= s - ad ? 1.0 : 0.0;
    st[FS_MAXLEN] = fmax(st[FS_MAXLEN], (double)(k1 - k0));
    st[FS_INF] = fmax(st[FS_INF], s);
    st[FS_DMAX] = fmax(st[FS_DMAX], ad);
    if (d != 0.0) {
      st[FS_RELOFF] += so / d;
      st[FS_RELOFF_N] += 1.0;
      st[FS_DMIN_NZ] = fmin(st[FS_DMIN_NZ], ad);
    }
  }
  __shared__ double red[FEAT_NT / 32][FEAT_STATS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < FEAT_STATS; ++k) {
    double v = st[k];
    for (int o = 16; o > 0; o >>= 1) v = fs_combine(k, v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < FEAT_STATS) {
    const int k = threadIdx.x;
    double v = red[0][k];
    for (int w = 1; w < FEAT_NT / 32; ++w) v = fs_combine(k, v, red[w][k]);
    part[(long long)blockIdx.x * FEAT_STATS + k] = v;
  }
}

__device__ __forceinline__ double lg30(double x) { return log10(fmax(x, 1e-30)); }

// Combines the G per-CTA statistics (one thread per statistic, CTA order) into the features.
__global__ void k_features_final(const double* __restrict__ part, int G, int n, long long nnz,
                                 float* __restrict__ f) {
  __shared__ double st[FEAT_STATS];
  const int k = threadIdx.x;
  if (k < FEAT_STATS) {
    double v = fs_identity(k);
    for (int b = 0; b < G; ++b) v = fs_combine(k, v, part[(long long)b * FEAT_STATS + k]);
    st[k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double dn = (double)n, dz = (double)(nnz > 0 ? nnz : 1);
    const double dmin = isinf(st[FS_DMIN_NZ]) ? 0.0 : st[FS_DMIN_NZ];
    const double v[SEL_NF] = {
        lg30(dn),
        lg30(dz),
        (double)nnz / dn,
        st[FS_MAXLEN],
        st[FS_RATIO] / dn,
        st[FS_RATIO_MIN],
        st[FS_DOM] / dn,
        lg30(st[FS_INF]),
        lg30(sqrt(st[FS_FRO2])),
        lg30(st[FS_AMAX]),
        lg30(st[FS_DABS] / dn),
        lg30(st[FS_DMAX]) - lg30(dmin),
        st[FS_DEN] > 0.0 ? st[FS_NUM] / st[FS_DEN] : 0.0,
        st[FS_RELOFF_N] > 0.0 ? st[FS_RELOFF] / st[FS_RELOFF_N] : 0.0,
        log10(1.0 + st[FS_DIST] / dz),
        log10(1.0 + st[FS_DISTMAX])};
    for (int q = 0; q < SEL_NF; ++q) f[q] = (float)v[q];
  }
}

// ---- MLP (flat weights: W1[16][64], b1[64], W2[64][64], b2[64], W3[64][32], b3[32]) ----
struct MlpLayout {
  static constexpr int W1 = 0, B1 = W1 + SEL_NF * SEL_NH, W2 = B1 + SEL_NH, B2 = W2 + SEL_NH * SEL_NH,
                       W3 = B2 + SEL_NH, B3 = W3 + SEL_NH * SEL_NC, N = B3 + SEL_NC;
};
static_assert(MlpLayout::N == SEL_NP, "selector parameter count");

// Y[s][o] = act(b[o] + sum_i X[s][i] W[i][o]), thread per (s, o).
__global__ void k_mlp_fwd(const float* __restrict__ X, int B, int nin, const float* __restrict__ W,
                          const float* __restrict__ bias, float* __restrict__ Y, int nout, int relu) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)B * nout) return;
  const int s = (int)(t / nout), o = (int)(t % nout);
  float acc = bias[o];
  for (int i = 0; i < nin; ++i) acc += X[(long long)s * nin + i] * W[i * nout + o];
  Y[t] = relu ? fmaxf(acc, 0.0f) : acc;
}

// Softmax of the logits, per-sample loss -log p[label], dZ = (p - onehot) / B (thread per
// sample).  labels == nullptr: probabilities only.
__global__ void k_softmax_xent(const float* __restrict__ Z, int B, const int* __restrict__ labels,
                               float* __restrict__ P, float* __restrict__ dZ, float* __restrict__ ls) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const float* z = Z + (long long)s * SEL_NC;
  float zmax = z[0];
  for (int c = 1; c < SEL_NC; ++c) zmax = fmaxf(zmax, z[c]);
  float e[SEL_NC], sum = 0.0f;
  for (int c = 0; c < SEL_NC; ++c) {
    e[c] = expf(z[c] - zmax);
    sum += e[c];
  }
  for (int c = 0; c < SEL_NC; ++c) {
    const float p = e[c] / sum;
    P[(long long)s * SEL_NC + c] = p;
    if (labels) dZ[(long long)s * SEL_NC + c] = (p - (c == labels[s] ? 1.0f : 0.0f)) / (float)B;
  }
  if (labels) ls[s] = -logf(P[(long long)s * SEL_NC + labels[s]]);
}

// loss = mean of the per-sample losses (one thread, sample order).
__global__ void k_loss_mean(const float* __restrict__ ls, int B, float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float s = 0.0f;
  for (int i = 0; i < B; ++i) s += ls[i];
  *loss = s / (float)B;
}

// dW[i][o] = sum_s X[s][i] dY[s][o] and db[o] = sum_s dY[s][o] (thread per output, sample order).
__global__ void k_mlp_bwd_w(const float* __restrict__ X, const float* __restrict__ dY, int B, int nin,
                            int nout, float* __restrict__ dW, float* __restrict__ db) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nin * nout) {
    const int i = t / nout, o = t % nout;
    float acc = 0.0f;
    for (int s = 0; s < B; ++s) acc += X[(long long)s * nin + i] * dY[(long long)s * nout + o];
    dW[t] = acc;
  } else if (t < nin * nout + nout) {
    const int o = t - nin * nout;
    float acc = 0.0f;
    for (int s = 0; s < B; ++s) acc += dY[(long long)s * nout + o];
    db[o] = acc;
  }
}

// dX[s][i] = (sum_o dY[s][o] W[i][o]) * (H[s][i] > 0): back through W and the ReLU that
// produced H (thread per (s, i)).
__global__ void k_mlp_bwd_x(const float* __restrict__ dY, const float* __restrict__ W,
                            const float* __restrict__ H, int B, int nin, int nout,
                            float* __restrict__ dX) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)B * nin) return;
  const int s = (int)(t / nin), i = (int)(t % nin);
  float acc = 0.0f;
  for (int o = 0; o < nout; ++o) acc += dY[(long long)s * nout + o] * W[i * nout + o];
  dX[t] = H[t] > 0.0f ? acc : 0.0f;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8); c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// Device buffers of one forward/backward pass over B samples.
struct MlpWork {
  int B = 0;
  float *X = nullptr, *H1 = nullptr, *H2 = nullptr, *Z = nullptr, *P = nullptr, *dZ = nullptr,
        *dH2 = nullptr, *dH1 = nullptr, *ls = nullptr, *loss = nullptr;
  float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  int* labels = nullptr;
};

static void mlp_free(MlpWork& w) {
  float* fs[] = {w.X, w.H1, w.H2, w.Z, w.P, w.dZ, w.dH2, w.dH1, w.ls, w.loss, w.params, w.grad, w.m, w.v};
  for (float* q : fs)
    if (q) cudaFree(q);
  if (w.labels) cudaFree(w.labels);
  w = MlpWork{};
}

static int mlp_alloc(MlpWork& w, int B, bool train) {
  w.B = B;
  auto al = [&](float** q, size_t cnt) { return CUDA_STATUS(cudaMalloc((void**)q, sizeof(float) * std::max<size_t>(cnt, 1))); };
  int e;
  if ((e = al(&w.X, (size_t)B * SEL_NF)) || (e = al(&w.H1, (size_t)B * SEL_NH)) ||
      (e = al(&w.H2, (size_t)B * SEL_NH)) || (e = al(&w.Z, (size_t)B * SEL_NC)) ||
      (e = al(&w.P, (size_t)B * SEL_NC)) || (e = al(&w.params, SEL_NP)))
    return e;
  if (!train) return GMRES_OK;
  if ((e = al(&w.dZ, (size_t)B * SEL_NC)) || (e = al(&w.dH2, (size_t)B * SEL_NH)) ||
      (e = al(&w.dH1, (size_t)B * SEL_NH)) || (e = al(&w.ls, B)) || (e = al(&w.loss, 1)) ||
      (e = al(&w.grad, SEL_NP)) || (e = al(&w.m, SEL_NP)) || (e = al(&w.v, SEL_NP)))
    return e;
  return CUDA_STATUS(cudaMalloc((void**)&w.labels, sizeof(int) * std::max(B, 1)));
}

static inline int blocks_for(long long cnt, int nt = 256) { return (int)std::max(1LL, (cnt + nt - 1) / nt); }

// Forward pass of w.X through w.params into w.P (and, with labels, loss and dZ).
static int mlp_forward(MlpWork& w, bool with_loss, cudaStream_t s) {
  using L = MlpLayout;
  const int B = w.B;
  k_mlp_fwd<<<blocks_for((long long)B * SEL_NH), 256, 0, s>>>(w.X, B, SEL_NF, w.params + L::W1, w.params + L::B1, w.H1, SEL_NH, 1);
  k_mlp_fwd<<<blocks_for((long long)B * SEL_NH), 256, 0, s>>>(w.H1, B, SEL_NH, w.params + L::W2, w.params + L::B2, w.H2, SEL_NH, 1);
  k_mlp_fwd<<<blocks_for((long long)B * SEL_NC), 256, 0, s>>>(w.H2, B, SEL_NH, w.params + L::W3, w.params + L::B3, w.Z, SEL_NC, 0);
  k_softmax_xent<<<blocks_for(B), 256, 0, s>>>(w.Z, B, with_loss ? w.labels : nullptr, w.P, w.dZ, w.ls);
  if (with_loss) k_loss_mean<<<1, 32, 0, s>>>(w.ls, B, w.loss);
  CK(cudaGetLastError());
  return GMRES_OK;
}

// Gradient of the mean cross-entropy into w.grad (after mlp_forward with the loss).
static int mlp_backward(MlpWork& w, cudaStream_t s) {
  using L = MlpLayout;
  const int B = w.B;
  k_mlp_bwd_w<<<blocks_for(SEL_NH * SEL_NC + SEL_NC), 256, 0, s>>>(w.H2, w.dZ, B, SEL_NH, SEL_NC, w.grad + L::W3, w.grad + L::B3);
  k_mlp_bwd_x<<<blocks_for((long long)B * SEL_NH), 256, 0, s>>>(w.dZ, w.params + L::W3, w.H2, B, SEL_NH, SEL_NC, w.dH2);
  k_mlp_bwd_w<<<blocks_for(SEL_NH * SEL_NH + SEL_NH), 256, 0, s>>>(w.H1, w.dH2, B, SEL_NH, SEL_NH, w.grad + L::W2, w.grad + L::B2);
  k_mlp_bwd_x<<<blocks_for((long long)B * SEL_NH), 256, 0, s>>>(w.dH2, w.params + L::W2, w.H1, B, SEL_NH, SEL_NH, w.dH1);
  k_mlp_bwd_w<<<blocks_for(SEL_NF * SEL_NH + SEL_NH), 256, 0, s>>>(w.X, w.dH1, B, SEL_NF, SEL_NH, w.grad + L::W1, w.grad + L::B1);
  CK(cudaGetLastError());
  return GMRES_OK;
}

static int mlp_upload(MlpWork& w, const float* params, const float* X, const int* labels, cudaStream_t s) {
  CK(cudaMemcpyAsync(w.params, params, sizeof(float) * SEL_NP, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.X, X, sizeof(float) * (size_t)w.B * SEL_NF, cudaMemcpyHostToDevice, s));
  if (labels) CK(cudaMemcpyAsync(w.labels, labels, sizeof(int) * (size_t)w.B, cudaMemcpyHostToDevice, s));
  return GMRES_OK;
}

static bool labels_ok(const int* labels, int B) {
  for (int i = 0; i < B; ++i)
    if (labels[i] < 0 || labels[i] >= SEL_NC) return false;
  return true;
}

}  // namespace gm

extern "C" {

int gmres_matrix_features(const gmres_csr* A, float* features, void* stream) {
  if (!features) return GMRES_ERR_INVALID;
  if (int e = gm::validate_csr(A)) return e;
  if (A->n == 0) return GMRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int G = (int)std::min<long long>(4LL * sms, (A->n + gm::FEAT_NT - 1) / gm::FEAT_NT);
  double* part = nullptr;
  float* f = nullptr;
  CK(cudaMallocAsync((void**)&part, sizeof(double) * gm::FEAT_STATS * G, s));
  int e = CUDA_STATUS(cudaMallocAsync((void**)&f, sizeof(float) * gm::SEL_NF, s));
  if (!e) {
    gm::k_features_partial<<<G, gm::FEAT_NT, 0, s>>>(A->row_ptr, A->col_idx, A->vals, A->n, part);
    gm::k_features_final<<<1, 32, 0, s>>>(part, G, A->n, (long long)A->nnz, f);
    e = CUDA_STATUS(cudaGetLastError());
  }
  if (!e) e = CUDA_STATUS(cudaMemcpyAsync(features, f, sizeof(float) * gm::SEL_NF, cudaMemcpyDeviceToHost, s));
  cudaFreeAsync(part, s);
  if (f) cudaFreeAsync(f, s);
  if (!e) e = CUDA_STATUS(cudaStreamSynchronize(s));
  return e;
}

int gmres_mlp_forward(const float* params, const float* X, int32_t nsamp, float* probs, void* stream) {
  if (!params || !X || !probs || nsamp < 1) return GMRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  gm::MlpWork w;
  int e = gm::mlp_alloc(w, nsamp, false);
  if (!e) e = gm::mlp_upload(w, params, X, nullptr, s);
  if (!e) e = gm::mlp_forward(w, false, s);
  if (!e) e = CUDA_STATUS(cudaMemcpyAsync(probs, w.P, sizeof(float) * (size_t)nsamp * gm::SEL_NC, cudaMemcpyDeviceToHost, s));
  if (!e) e = CUDA_STATUS(cudaStreamSynchronize(s));
  cudaStreamSynchronize(s);
  gm::mlp_free(w);
  return e;
}

int gmres_mlp_loss_grad(const float* params, const float* X, const int32_t* labels, int32_t nsamp,
                        float* loss, float* grad, void* stream) {
  if (!params || !X || !labels || !loss || !grad || nsamp < 1) return GMRES_ERR_INVALID;
  if (!gm::labels_ok(labels, nsamp)) return GMRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  gm::MlpWork w;
  int e = gm::mlp_alloc(w, nsamp, true);
  if (!e) e = gm::mlp_upload(w, params, X, labels, s);
  if (!e) e = gm::mlp_forward(w, true, s);
  if (!e) e = gm::mlp_backward(w, s);
  if (!e) e = CUDA_STATUS(cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  if (!e) e = CUDA_STATUS(cudaMemcpyAsync(grad, w.grad, sizeof(float) * gm::SEL_NP, cudaMemcpyDeviceToHost, s));
  if (!e) e = CUDA_STATUS(cudaStreamSynchronize(s));
  cudaStreamSynchronize(s);
  gm::mlp_free(w);
  return e;
}

int gmres_mlp_train(float* params, const float* X, const int32_t* labels, int32_t nsamp, int32_t epochs,
                    float lr, float* losses, void* stream) {
  if (!params || !X || !labels || nsamp < 1 || epochs < 0 || !(lr > 0.0f)) return GMRES_ERR_INVALID;
  if (!gm::labels_ok(labels, nsamp)) return GMRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  gm::MlpWork w;
  int e = gm::mlp_alloc(w, nsamp, true);
  float* d_losses = nullptr;
  if (!e) e = CUDA_STATUS(cudaMalloc((void**)&d_losses, sizeof(float) * std::max(epochs, 1)));
  if (!e) e = gm::mlp_upload(w, params, X, labels, s);
  if (!e) e = CUDA_STATUS(cudaMemsetAsync(w.m, 0, sizeof(float) * gm::SEL_NP, s));
  if (!e) e = CUDA_STATUS(cudaMemsetAsync(w.v, 0, sizeof(float) * gm::SEL_NP, s));
  double b1t = 1.0, b2t = 1.0;
  for (int t = 1; !e && t <= epochs; ++t) {
    e = gm::mlp_forward(w, true, s);
    if (!e) e = CUDA_STATUS(cudaMemcpyAsync(d_losses + t - 1, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (!e) e = gm::mlp_backward(w, s);
    b1t *= 0.9;
    b2t *= 0.999;
    if (!e) {
      gm::k_adam<<<gm::blocks_for(gm::SEL_NP), 256, 0, s>>>(w.params, w.grad, w.m, w.v, gm::SEL_NP, lr,
                                                          (float)(1.0 - b1t), (float)(1.0 - b2t));
      e = CUDA_STATUS(cudaGetLastError());
    }
  }
  if (!e) e = CUDA_STATUS(cudaMemcpyAsync(params, w.params, sizeof(float) * gm::SEL_NP, cudaMemcpyDeviceToHost, s));
  if (!e && losses && epochs > 0)
    e = CUDA_STATUS(cudaMemcpyAsync(losses, d_losses, sizeof(float) * epochs, cudaMemcpyDeviceToHost, s));
  if (!e) e = CUDA_STATUS(cudaStreamSynchronize(s));
  cudaStreamSynchronize(s);
  if (d_losses) cudaFree(d_losses);
  gm::mlp_free(w);
  return e;
}

int gmres_select_params(const gmres_csr* A, const gmres_selector* sel, gmres_params* p,
                        int32_t* class_out, float* confidence_out, void* stream) {
  if (!A || !p) return GMRES_ERR_INVALID;
  // the fixed default, also the fallback
  p->restart_m = 50;
  p->poly_degree = 0;
  p->inner_prec = GMRES_FP32;
  p->inner_rtol = 1e-4;
  if (class_out) *class_out = -1;
  if (confidence_out) *confidence_out = 0.0f;
  if (!sel || !sel->params) return GMRES_OK;
  if (!sel->feat_mean || !sel->feat_scale || !sel->class_m || !sel->class_degree ||
      !sel->class_prec || !sel->class_inner_rtol)
    return GMRES_ERR_INVALID;
  float f[GMRES_SEL_FEATURES];
  if (int e = gmres_matrix_features(A, f, stream)) return e;
  for (int i = 0; i < GMRES_SEL_FEATURES; ++i) f[i] = (f[i] - sel->feat_mean[i]) * sel->feat_scale[i];
  float prob[GMRES_SEL_CLASSES];
  if (int e = gmres_mlp_forward(sel->params, f, 1, prob, stream)) return e;
  int best = 0;
  for (int c = 1; c < GMRES_SEL_CLASSES; ++c)
    if (prob[c] > prob[best]) best = c;
  if (confidence_out) *confidence_out = prob[best];
  if (!(prob[best] >= sel->min_confidence)) return GMRES_OK;
  gmres_params q = *p;
  q.restart_m = sel->class_m[best];
  q.poly_degree = sel->class_degree[best];
  q.inner_prec = sel->class_prec[best];
  q.inner_rtol = sel->class_inner_rtol[best];
  if (gm::validate_params(&q)) return GMRES_OK;  // a malformed class entry: keep the default
  *p = q;
  if (class_out) *class_out = best;
  return GMRES_OK;
}

}  // extern "C"
