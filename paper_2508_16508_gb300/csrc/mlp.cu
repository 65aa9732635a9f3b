// Capacity predictor: a small FP32 MLP (n_in -> hidden x layers -> n_out, ReLU)
// trained with a pinball (quantile) loss and Adam, plus the capacity sizing
// that turns its prediction into per-model slab capacities. The paper has no
// learned component; its Section 4 notes that the maximum number of agents
// must be known in advance, which is what this predicts.
//
// Everything is plain FP32 FFMA with shared-memory tiles: the matrices are at
// most 128 wide, so tensor cores would idle on the operand staging.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace abm {

constexpr int kGT = 64;   // GEMM tile (rows and columns)
constexpr int kGK = 16;   // GEMM k-step
constexpr int kGThreads = 256;

// C[m][n] (+)= sum_k opA(m,k) * opB(k,n), with opA(m,k) = TA ? A[k*lda + m] : A[m*lda + k]
// and opB(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]. Epilogue: + bias[n], ReLU,
// or multiply by (mask[m*ldm + n] > 0). Rows of A may be gathered through an
// affine permutation of [0, rows): row(m) = (pa * (m0 + m) + pc) % rows.
struct GemmArgs {
  int M, N, K;
  const float* A;
  int lda;
  const float* B;
  int ldb;
  float* C;
  int ldc;
  const float* bias;
  const float* mask;
  int ldm;
  int relu;
  // optional row gather of A (only when !TA): 0 = none
  long long gather_rows, gather_a, gather_c, gather_m0;
  // split-K: grid.z slices of K, each writing its own C slice (C + z * split_stride)
  int k_per_split;
  long long split_stride;
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(kGThreads) k_gemm(GemmArgs g) {
  __shared__ float sA[kGK][kGT + 4];
  __shared__ float sB[kGK][kGT + 4];
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
  const int kbeg = blockIdx.z * g.k_per_split;
  const int kend = min(g.K, kbeg + g.k_per_split);
  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += kGK) {
    // stage A tile (kGK x kGT) and B tile (kGK x kGT)
    for (int i = threadIdx.x; i < kGK * kGT; i += kGThreads) {
      const int kk = i / kGT, mm = i % kGT;
      const int m = m0 + mm, k = k0 + kk;
      float va = 0.f;
      if (m < g.M && k < kend) {
        if (TA) {
          va = g.A[(size_t)k * g.lda + m];
        } else {
          long long row = m;
          if (g.gather_rows) row = (g.gather_a * (g.gather_m0 + m) + g.gather_c) % g.gather_rows;
          va = g.A[(size_t)row * g.lda + k];
        }
      }
      sA[kk][mm] = va;
      const int n = n0 + mm;
      float vb = 0.f;
      if (n < g.N && k < kend) vb = TB ? g.B[(size_t)n * g.ldb + k] : g.B[(size_t)k * g.ldb + n];
      sB[kk][mm] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* C = g.C + (size_t)blockIdx.z * g.split_stride;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      float v = acc[i][j];
      if (g.bias) v += g.bias[n];
      if (g.relu) v = fmaxf(v, 0.f);
      if (g.mask && !(g.mask[(size_t)m * g.ldm + n] > 0.f)) v = 0.f;
      C[(size_t)m * g.ldc + n] = v;
    }
  }
}

// out[i] = sum over z of part[z * stride + i] (fixed order: deterministic)
__global__ void k_sum_splits(const float* part, int nsplit, long long stride, int n, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < nsplit; ++z) s += part[(size_t)z * stride + i];
    out[i] = s;
  }
}

// column sums of a [rows x cols] matrix, one thread per column, fixed order
__global__ void k_colsum(const float* d, int rows, int cols, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += d[(size_t)r * cols + c];
  out[c] = s;
}

// pinball loss at quantile tau: e = y - yhat, loss = max(tau e, (tau - 1) e),
// averaged over all entries; dyhat = d loss / d yhat. Targets are gathered
// with the same row permutation as the inputs.
__global__ void k_pinball(const float* yhat, const float* y, int B, int n_out, float tau, long long grows,
                          long long ga, long long gc, long long gm0, float* dyhat, float* loss_part) {
  __shared__ float s[256];
  float acc = 0.f;
  const float scale = 1.f / (float)(B * n_out);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * n_out; i += gridDim.x * blockDim.x) {
    const int r = i / n_out, o = i % n_out;
    long long row = r;
    if (grows) row = (ga * (gm0 + r) + gc) % grows;
    const float e = y[(size_t)row * n_out + o] - yhat[i];
    acc += e > 0.f ? tau * e : (tau - 1.f) * e;
    dyhat[i] = (e > 0.f ? -tau : 1.f - tau) * scale;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = s[0];
}

__global__ void k_loss_final(const float* part, int n, float scale, float* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s * scale;
  }
}

// Adam (Kingma & Ba, 2015) with bias correction
__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    p[i] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// He-uniform initialisation from Philox: W ~ U(-sqrt(6/fan_in), +sqrt(6/fan_in)), b = 0
__global__ void k_mlp_init(float* p, long long n, const long long* off, const int* fan_in, int nlayers, u32 seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int l = 0;
    while (l + 1 < 2 * nlayers && off[l + 1] <= i) ++l;
    if (l & 1) {  // bias block
      p[i] = 0.f;
    } else {
      const u32 u = draw(seed, 0x4D4C50u, (u32)(i >> 32), (u32)i, 15u, (u32)l);
      const float r = ((float)(u >> 8) + 0.5f) * (1.f / 16777216.f);  // (0, 1)
      const float lim = sqrtf(6.f / (float)fan_in[l >> 1]);
      p[i] = (2.f * r - 1.f) * lim;
    }
  }
}

// features of a model: log1p(side), log1p(n0 sheep), log1p(n0 wolves), the 8
// rule params over their nominal values, horizon / 500
__global__ void k_features(const int32_t* tab, int B, const int32_t* nominal, float* x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
    const int32_t* t = tab + (size_t)i * 12;
    float* o = x + (size_t)i * 12;
    o[0] = log1pf((float)t[0]);
    o[1] = log1pf((float)t[1]);
    o[2] = log1pf((float)t[2]);
    for (int j = 0; j < 8; ++j) o[3 + j] = (float)(u32)t[3 + j] / (float)(u32)nominal[j];
    o[11] = (float)t[11] / 500.f;
  }
}

// capacity from a predicted log peak: min(cap_max, roundup(ceil(exp(yhat) * (1 + margin)), round_to)),
// never below the initial population and never below round_to
__global__ void k_capacity(const float* yhat, int B, float margin, int round_to, const int32_t* cap_max,
                           const int32_t* n0, int32_t* cap) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * B; i += gridDim.x * blockDim.x) {
    const double want = ceil(exp((double)yhat[i]) * (1.0 + (double)margin));
    long long c = (long long)fmin(want, 2147483647.0);
    if (c < n0[i]) c = n0[i];
    c = ((c + round_to - 1) / round_to) * round_to;
    if (c < round_to) c = round_to;
    if (c > cap_max[i]) c = cap_max[i];
    cap[i] = (int32_t)c;
  }
}

}  // namespace abm

// ============================================================================
using namespace abm;

struct abm_mlp {
  int n_in, hidden, layers, n_out, max_batch;  // layers = hidden layers
  int nlin;                                    // linear maps = layers + 1
  std::vector<int> din, dout;
  std::vector<long long> offW, offb;
  long long nparams;
  float *p, *g, *m, *v;
  float* act;    // activations: [nlin + 1] blocks of max_batch x width
  std::vector<long long> offA;
  float* dact;   // gradients of activations, same layout
  float* part;   // split-K partials
  float* lossp;  // loss partial sums
  long long* d_off;
  int* d_fan;
  int adam_t;
};

static void mlp_free(abm_mlp* n) {
  cudaFree(n->p);
  cudaFree(n->g);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->act);
  cudaFree(n->dact);
  cudaFree(n->part);
  cudaFree(n->lossp);
  cudaFree(n->d_off);
  cudaFree(n->d_fan);
  delete n;
}

static const int kSplits = 32;

extern "C" abm_status abm_mlp_destroy(abm_mlp* n) {
  if (!n) return ABM_ERR_ARG;
  mlp_free(n);
  return ABM_OK;
}

extern "C" abm_status abm_mlp_create(int32_t n_in, int32_t hidden, int32_t layers, int32_t n_out, uint32_t seed,
                                     int32_t max_batch, void* stream, abm_mlp** out) {
  if (!out || n_in < 1 || n_in > 1024 || hidden < 1 || hidden > 1024 || layers < 1 || layers > 8 || n_out < 1 ||
      n_out > 1024 || max_batch < 1)
    return ABM_ERR_ARG;
  abm_mlp* n = new (std::nothrow) abm_mlp();
  if (!n) return ABM_ERR_OOM;
  n->n_in = n_in;
  n->hidden = hidden;
  n->layers = layers;
  n->n_out = n_out;
  n->max_batch = max_batch;
  n->nlin = layers + 1;
  long long off = 0;
  std::vector<long long> offs;
  std::vector<int> fan;
  for (int l = 0; l < n->nlin; ++l) {
    const int di = l == 0 ? n_in : hidden, dd = l == n->nlin - 1 ? n_out : hidden;
    n->din.push_back(di);
    n->dout.push_back(dd);
    n->offW.push_back(off);
    offs.push_back(off);
    off += (long long)di * dd;
    n->offb.push_back(off);
    offs.push_back(off);
    off += dd;
    fan.push_back(di);
  }
  n->nparams = off;
  long long aoff = 0;
  for (int l = 0; l <= n->nlin; ++l) {
    n->offA.push_back(aoff);
    const int w = l == 0 ? n_in : n->dout[l - 1];
    aoff += (long long)max_batch * w;
  }
  const size_t P = (size_t)n->nparams;
  bool ok = cudaMalloc(&n->p, P * 4) == cudaSuccess && cudaMalloc(&n->g, P * 4) == cudaSuccess &&
            cudaMalloc(&n->m, P * 4) == cudaSuccess && cudaMalloc(&n->v, P * 4) == cudaSuccess &&
            cudaMalloc(&n->act, (size_t)aoff * 4) == cudaSuccess && cudaMalloc(&n->dact, (size_t)aoff * 4) == cudaSuccess &&
            cudaMalloc(&n->part, (size_t)kSplits * std::max(hidden, n_in) * std::max(hidden, n_out) * 4) == cudaSuccess &&
            cudaMalloc(&n->lossp, 1024 * 4) == cudaSuccess &&
            cudaMalloc(&n->d_off, offs.size() * sizeof(long long)) == cudaSuccess &&
            cudaMalloc(&n->d_fan, fan.size() * sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mlp_free(n);
    return ABM_ERR_OOM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(n->d_off, offs.data(), offs.size() * sizeof(long long), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(n->d_fan, fan.data(), fan.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(n->m, 0, P * 4, st) != cudaSuccess || cudaMemsetAsync(n->v, 0, P * 4, st) != cudaSuccess) {
    mlp_free(n);
    return ABM_ERR_CUDA;
  }
  k_mlp_init<<<num_sms() * 4, 256, 0, st>>>(n->p, n->nparams, n->d_off, n->d_fan, n->nlin, seed);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    mlp_free(n);
    return ABM_ERR_CUDA;
  }
  n->adam_t = 0;
  *out = n;
  return ABM_OK;
}

template <bool TA, bool TB>
static void gemm(const GemmArgs& a, cudaStream_t st, int splits = 1) {
  dim3 grid((unsigned)((a.N + kGT - 1) / kGT), (unsigned)((a.M + kGT - 1) / kGT), (unsigned)splits);
  k_gemm<TA, TB><<<grid, kGThreads, 0, st>>>(a);
}

static GemmArgs gargs(int M, int N, int K) {
  GemmArgs a;
  std::memset(&a, 0, sizeof(a));
  a.M = M;
  a.N = N;
  a.K = K;
  a.k_per_split = K;
  return a;
}

struct Perm {
  long long rows, a, c, m0;
};

// forward through all layers; the output lands in act block nlin
static abm_status mlp_forward(abm_mlp* n, const float* x, int B, const Perm& pm, cudaStream_t st) {
  for (int l = 0; l < n->nlin; ++l) {
    GemmArgs a = gargs(B, n->dout[l], n->din[l]);
    if (l == 0) {
      a.A = x;
      a.gather_rows = pm.rows;
      a.gather_a = pm.a;
      a.gather_c = pm.c;
      a.gather_m0 = pm.m0;
    } else {
      a.A = n->act + n->offA[l];
    }
    a.lda = n->din[l];
    a.B = n->p + n->offW[l];
    a.ldb = n->dout[l];
    a.C = n->act + n->offA[l + 1];
    a.ldc = n->dout[l];
    a.bias = n->p + n->offb[l];
    a.relu = l < n->nlin - 1;
    gemm<false, false>(a, st);
  }
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

// loss + gradients of all parameters into n->g (loss_out: device float, nullable)
static abm_status mlp_backward(abm_mlp* n, const float* x, const float* y, int B, float tau, const Perm& pm,
                               float* loss_out, cudaStream_t st) {
  const int L = n->nlin;
  const int nblk = std::min(1024, std::max(1, (B * n->n_out + 255) / 256));
  k_pinball<<<nblk, 256, 0, st>>>(n->act + n->offA[L], y, B, n->n_out, tau, pm.rows, pm.a, pm.c, pm.m0,
                                  n->dact + n->offA[L], n->lossp);
  if (loss_out) k_loss_final<<<1, 32, 0, st>>>(n->lossp, nblk, 1.f / (float)(B * n->n_out), loss_out);
  for (int l = L - 1; l >= 0; --l) {
    const float* dY = n->dact + n->offA[l + 1];  // [B x dout]
    // dW = X^T dY  (din x dout), split over the batch, summed in fixed order
    const int per = (((B + kSplits - 1) / kSplits) + kGK - 1) / kGK * kGK;
    const int splits = (B + per - 1) / per;
    GemmArgs a = gargs(n->din[l], n->dout[l], B);
    a.A = n->act + n->offA[l];  // block 0 holds the gathered input rows
    a.lda = n->din[l];
    a.B = dY;
    a.ldb = n->dout[l];
    a.C = n->part;
    a.ldc = n->dout[l];
    a.k_per_split = per;
    a.split_stride = (long long)n->din[l] * n->dout[l];
    gemm<true, false>(a, st, splits);
    k_sum_splits<<<std::max(1, std::min(256, (n->din[l] * n->dout[l] + 255) / 256)), 256, 0, st>>>(
        n->part, splits, a.split_stride, n->din[l] * n->dout[l], n->g + n->offW[l]);
    k_colsum<<<(n->dout[l] + 127) / 128, 128, 0, st>>>(dY, B, n->dout[l], n->g + n->offb[l]);
    if (l > 0) {
      // dX = (dY W^T) * (X > 0)
      GemmArgs d = gargs(B, n->din[l], n->dout[l]);
      d.A = dY;
      d.lda = n->dout[l];
      d.B = n->p + n->offW[l];
      d.ldb = n->dout[l];
      d.C = n->dact + n->offA[l];
      d.ldc = n->din[l];
      d.mask = n->act + n->offA[l];
      d.ldm = n->din[l];
      gemm<false, true>(d, st);
    }
  }
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

// copy the (gathered) input rows into act block 0 so that the first layer's
// weight gradient can read them transposed
__global__ void k_gather_rows(const float* x, int B, int w, long long rows, long long ga, long long gc, long long gm0,
                              float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * w; i += gridDim.x * blockDim.x) {
    const int r = i / w, c = i % w;
    long long row = r;
    if (rows) row = (ga * (gm0 + r) + gc) % rows;
    out[i] = x[(size_t)row * w + c];
  }
}

static Perm make_perm(int64_t rows, int64_t a, int64_t c, int64_t m0) {
  Perm p;
  p.rows = rows;
  p.a = a;
  p.c = c;
  p.m0 = m0;
  return p;
}

extern "C" abm_status abm_mlp_forward(abm_mlp* n, const float* x, int32_t B, float* y, void* stream) {
  if (!n || !x || !y || B < 1 || B > n->max_batch) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  abm_status e = mlp_forward(n, x, B, make_perm(0, 0, 0, 0), st);
  if (e != ABM_OK) return e;
  ABM_CUDA_TRY(cudaMemcpyAsync(y, n->act + n->offA[n->nlin], sizeof(float) * (size_t)B * n->n_out,
                               cudaMemcpyDeviceToDevice, st));
  return ABM_OK;
}

extern "C" abm_status abm_mlp_gradients(abm_mlp* n, const float* x, const float* y, int32_t B, float tau,
                                        int64_t perm_rows, int64_t perm_a, int64_t perm_c, int64_t perm_m0,
                                        float* loss_out, void* stream) {
  if (!n || !x || !y || B < 1 || B > n->max_batch || perm_rows < 0 || (perm_rows > 0 && perm_a < 1)) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const Perm pm = make_perm(perm_rows, perm_a, perm_c, perm_m0);
  abm_status e = mlp_forward(n, x, B, pm, st);
  if (e != ABM_OK) return e;
  k_gather_rows<<<std::max(1, std::min(1024, (B * n->n_in + 255) / 256)), 256, 0, st>>>(
      x, B, n->n_in, pm.rows, pm.a, pm.c, pm.m0, n->act);
  return mlp_backward(n, x, y, B, tau, pm, loss_out, st);
}

extern "C" abm_status abm_mlp_train_step(abm_mlp* n, const float* x, const float* y, int32_t B, float tau, float lr,
                                         int64_t perm_rows, int64_t perm_a, int64_t perm_c, int64_t perm_m0,
                                         float* loss_out, void* stream) {
  abm_status e = abm_mlp_gradients(n, x, y, B, tau, perm_rows, perm_a, perm_c, perm_m0, loss_out, stream);
  if (e != ABM_OK) return e;
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - std::pow((double)b1, n->adam_t));
  const float c2 = (float)(1.0 - std::pow((double)b2, n->adam_t));
  k_adam<<<std::max(1, std::min(1024, (int)((n->nparams + 255) / 256))), 256, 0, (cudaStream_t)stream>>>(
      n->p, n->g, n->m, n->v, (int)n->nparams, lr, b1, b2, eps, c1, c2);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_mlp_params(abm_mlp* n, float** params, float** grads, int64_t* count) {
  if (!n) return ABM_ERR_ARG;
  if (params) *params = n->p;
  if (grads) *grads = n->g;
  if (count) *count = n->nparams;
  return ABM_OK;
}

extern "C" abm_status abm_mlp_set_params(abm_mlp* n, const float* src, int64_t count, void* stream) {
  if (!n || !src || count != n->nparams) return ABM_ERR_ARG;
  ABM_CUDA_TRY(cudaMemcpyAsync(n->p, src, sizeof(float) * (size_t)count, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  return ABM_OK;
}

extern "C" abm_status abm_mlp_get_params(abm_mlp* n, float* dst, int64_t count, void* stream) {
  if (!n || !dst || count != n->nparams) return ABM_ERR_ARG;
  ABM_CUDA_TRY(cudaMemcpyAsync(dst, n->p, sizeof(float) * (size_t)count, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  return ABM_OK;
}

extern "C" abm_status abm_mlp_get_grads(abm_mlp* n, float* dst, int64_t count, void* stream) {
  if (!n || !dst || count != n->nparams) return ABM_ERR_ARG;
  ABM_CUDA_TRY(cudaMemcpyAsync(dst, n->g, sizeof(float) * (size_t)count, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  return ABM_OK;
}

extern "C" abm_status abm_mlp_reset_adam(abm_mlp* n, void* stream) {
  if (!n) return ABM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ABM_CUDA_TRY(cudaMemsetAsync(n->m, 0, sizeof(float) * (size_t)n->nparams, st));
  ABM_CUDA_TRY(cudaMemsetAsync(n->v, 0, sizeof(float) * (size_t)n->nparams, st));
  n->adam_t = 0;
  return ABM_OK;
}

extern "C" abm_status abm_capacity_features(const int32_t* table, int32_t B, const int32_t* nominal, float* x,
                                            void* stream) {
  if (!table || !nominal || !x || B < 1) return ABM_ERR_ARG;
  k_features<<<std::max(1, std::min(1024, (B + 255) / 256)), 256, 0, (cudaStream_t)stream>>>(table, B, nominal, x);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}

extern "C" abm_status abm_capacity_from_prediction(const float* yhat, int32_t B, float margin, int32_t round_to,
                                                   const int32_t* cap_max, const int32_t* n0, int32_t* cap,
                                                   void* stream) {
  if (!yhat || !cap_max || !n0 || !cap || B < 1 || round_to < 1 || margin < 0.f) return ABM_ERR_ARG;
  k_capacity<<<std::max(1, std::min(1024, (2 * B + 255) / 256)), 256, 0, (cudaStream_t)stream>>>(
      yhat, B, margin, round_to, cap_max, n0, cap);
  ABM_LAUNCH_CHECK();
  return ABM_OK;
}
