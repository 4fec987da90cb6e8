// Training of the learned blending coefficient on the GPU: the network maps
// an element's normalised modal energies (encoded, nin inputs) through two
// hidden layers of 32 ReLU units to a sigmoid output; the loss is the
// cross-entropy against the smoothness indicator's alpha (in [0, 1], taken as
// a probability), whose gradient in the output logit is (y - t) / n.  Forward and
// backward passes, Adam, and the epoch loop are this file's kernels.
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/cr.h"
#include "cr_common.cuh"

namespace {

constexpr int kH = 32;
constexpr int kChunk = 64;    // samples cached in shared memory per pass
constexpr int kThreads = 128;

__host__ __device__ constexpr int param_count(int nin) {
  return kH * nin + kH + kH * kH + kH + kH + 1;
}

// Gradient of the cross-entropy over samples [0, n) (indices through idx
// when given) and the loss (t softplus(-z) + (1 - t) softplus(z)) * inv_n.
// One block handles chunks of 64 samples: threads 0..63 run forward and
// backward for one sample each into shared memory, then all threads reduce
// their share of the gradient entries.  Block b writes its partial sums to
// part[b][0..P) and its loss to part[b][P]; k_mlp_reduce adds the blocks in a
// fixed order, so the result does not depend on block scheduling.
template <int NIN>
__global__ void __launch_bounds__(kThreads) k_mlp_grad(const float* __restrict__ prm,
                                                        const float* __restrict__ X,
                                                        const float* __restrict__ T,
                                                        const int* __restrict__ idx, int n,
                                                        float inv_n, float* __restrict__ part) {
  constexpr int P = param_count(NIN);
  constexpr int PER = (P + kThreads - 1) / kThreads;
  constexpr int REC = NIN + 4 * kH + 1;  // x, h1, da1, h2, da2, dz per sample
  extern __shared__ float sm[];
  float* sp = sm;                // parameters [P]
  float* sr = sm + P;            // sample records [kChunk][REC]
  const int tid = threadIdx.x;
  for (int g = tid; g < P; g += kThreads) sp[g] = prm[g];
  const float* W1 = sp;
  const float* B1 = W1 + kH * NIN;
  const float* W2 = B1 + kH;
  const float* B2 = W2 + kH * kH;
  const float* W3 = B2 + kH;
  float acc[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) acc[r] = 0.0f;
  float lsum = 0.0f;
  __syncthreads();
  const float B3 = W3[kH];  // read only after every thread's copy is visible
  for (int base = blockIdx.x * kChunk; base < n; base += gridDim.x * kChunk) {
    const int cnt = min(kChunk, n - base);
    if (tid < cnt) {
      const int s = idx ? idx[base + tid] : base + tid;
      float* R = sr + tid * REC;
      float* x = R;
      float* h1 = x + NIN;
      float* d1 = h1 + kH;
      float* h2 = d1 + kH;
      float* d2 = h2 + kH;
#pragma unroll
      for (int i = 0; i < NIN; ++i) x[i] = X[(size_t)s * NIN + i];
      for (int j = 0; j < kH; ++j) {
        float a = B1[j];
#pragma unroll
        for (int i = 0; i < NIN; ++i) a += W1[j * NIN + i] * x[i];
        h1[j] = a;  // pre-activation kept until the backward pass
      }
      float z = B3;
      for (int j = 0; j < kH; ++j) {
        float a = B2[j];
        for (int i = 0; i < kH; ++i) a += W2[j * kH + i] * fmaxf(h1[i], 0.0f);
        h2[j] = a;
        z += W3[j] * fmaxf(a, 0.0f);
      }
      const float y = 1.0f / (1.0f + expf(-z));
      const float t = T[s];
      const float sp = log1pf(expf(-fabsf(z)));  // softplus(z) = max(z, 0) + sp
      lsum += (t * (fmaxf(-z, 0.0f) + sp) + (1.0f - t) * (fmaxf(z, 0.0f) + sp)) * inv_n;
      const float dz = (y - t) * inv_n;
      R[REC - 1] = dz;
      for (int j = 0; j < kH; ++j) d2[j] = h2[j] > 0.0f ? dz * W3[j] : 0.0f;
      for (int i = 0; i < kH; ++i) {
        float a = 0.0f;
        for (int j = 0; j < kH; ++j) a += W2[j * kH + i] * d2[j];
        d1[i] = h1[i] > 0.0f ? a : 0.0f;
      }
      for (int j = 0; j < kH; ++j) {
        h1[j] = fmaxf(h1[j], 0.0f);
        h2[j] = fmaxf(h2[j], 0.0f);
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int g = tid + r * kThreads;
      if (g >= P) break;
      float a = 0.0f;
      if (g < kH * NIN) {  // W1[j][i] += d1[j] x[i]
        const int j = g / NIN, i = g - j * NIN;
        for (int s = 0; s < cnt; ++s) a += sr[s * REC + NIN + kH + j] * sr[s * REC + i];
      } else if (g < kH * NIN + kH) {  // b1
        const int j = g - kH * NIN;
        for (int s = 0; s < cnt; ++s) a += sr[s * REC + NIN + kH + j];
      } else if (g < kH * NIN + kH + kH * kH) {  // W2[j][i] += d2[j] h1[i]
        const int gg = g - kH * NIN - kH, j = gg / kH, i = gg - j * kH;
        for (int s = 0; s < cnt; ++s) a += sr[s * REC + NIN + 3 * kH + j] * sr[s * REC + NIN + i];
      } else if (g < kH * NIN + 2 * kH + kH * kH) {  // b2
        const int j = g - kH * NIN - kH - kH * kH;
        for (int s = 0; s < cnt; ++s) a += sr[s * REC + NIN + 3 * kH + j];
      } else if (g < P - 1) {  // w3[j] += dz h2[j]
        const int j = g - kH * NIN - 2 * kH - kH * kH;
        for (int s = 0; s < cnt; ++s) a += sr[s * REC + REC - 1] * sr[s * REC + NIN + 2 * kH + j];
      } else {  // b3
        for (int s = 0; s < cnt; ++s) a += sr[s * REC + REC - 1];
      }
      acc[r] += a;
    }
    __syncthreads();
  }
  float* out = part + (size_t)blockIdx.x * (P + 1);
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int g = tid + r * kThreads;
    if (g < P) out[g] = acc[r];
  }
  // block sum of the per-sample losses (threads >= 64 hold 0), fixed order
  __syncthreads();
  sr[tid] = lsum;
  __syncthreads();
  if (tid == 0) {
    float l = 0.0f;
    for (int i = 0; i < kThreads; ++i) l += sr[i];
    out[P] = l;
  }
}

// grad[g] = sum over blocks b = 0, 1, ... of part[b][g]; loss likewise (g = P).
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblocks, int P,
                             float* __restrict__ grad, float* __restrict__ loss) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > P) return;
  float a = 0.0f;
  for (int b = 0; b < nblocks; ++b) a += part[(size_t)b * (P + 1) + g];
  if (g < P) grad[g] = a;
  else *loss = a;
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f;
  const float mi = b1 * m[i] + (1.0f - b1) * g[i];
  const float vi = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void k_accumulate(float* dst, const float* src) { *dst += *src; }

constexpr int kMaxGradBlocks = 304;  // two blocks per SM

int grad_blocks(int n) {
  int blocks = (n + kChunk - 1) / kChunk;
  if (blocks > kMaxGradBlocks) blocks = kMaxGradBlocks;
  return blocks < 1 ? 1 : blocks;
}

// Loss and gradient of samples [0, n) into grad and loss (overwritten); part
// is scratch of grad_blocks(n) * (P + 1) floats.
template <int NIN>
cudaError_t launch_grad(const float* prm, const float* X, const float* T, const int* idx, int n,
                        float* part, float* grad, float* loss, cudaStream_t s) {
  constexpr int P = param_count(NIN);
  const size_t smem = (size_t)(P + kChunk * (NIN + 4 * kH + 1)) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad<NIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = grad_blocks(n);
  k_mlp_grad<NIN><<<blocks, kThreads, smem, s>>>(prm, X, T, idx, n, 1.0f / float(n), part);
  k_mlp_reduce<<<(P + 1 + 255) / 256, 256, 0, s>>>(part, blocks, P, grad, loss);
  return cudaGetLastError();
}

cudaError_t dispatch_grad(int nin, const float* prm, const float* X, const float* T, const int* idx,
                          int n, float* part, float* grad, float* loss, cudaStream_t s) {
  switch (nin) {
    case 2: return launch_grad<2>(prm, X, T, idx, n, part, grad, loss, s);
    case 3: return launch_grad<3>(prm, X, T, idx, n, part, grad, loss, s);
    case 4: return launch_grad<4>(prm, X, T, idx, n, part, grad, loss, s);
    case 5: return launch_grad<5>(prm, X, T, idx, n, part, grad, loss, s);
    case 9: return launch_grad<9>(prm, X, T, idx, n, part, grad, loss, s);
    case 16: return launch_grad<16>(prm, X, T, idx, n, part, grad, loss, s);
    case 25: return launch_grad<25>(prm, X, T, idx, n, part, grad, loss, s);
  }
  return cudaErrorInvalidValue;
}

bool nin_supported(int nin) {
  return nin == 2 || nin == 3 || nin == 4 || nin == 5 || nin == 9 || nin == 16 || nin == 25;
}

uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int cr_mlp_param_count(int nin) { return nin_supported(nin) ? param_count(nin) : -1; }

cr_status cr_mlp_grad(int nin, const float* params, const float* X, const float* t, int n,
                      float* grad, float* loss, void* stream) {
  if (!nin_supported(nin) || !params || !X || !t || !grad || !loss || n < 1) return CR_E_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = nullptr;  // per-block partial sums, stream-ordered allocation
  const size_t bytes = sizeof(float) * (size_t)grad_blocks(n) * (param_count(nin) + 1);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&part), bytes, s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CR_E_NOMEM : CR_E_CUDA;
  e = dispatch_grad(nin, params, X, t, nullptr, n, part, grad, loss, s);
  const cudaError_t e2 = cudaFreeAsync(part, s);
  return (e == cudaSuccess && e2 == cudaSuccess) ? CR_OK : CR_E_CUDA;
}

cr_status cr_mlp_train(int nin, float* params, const float* X, const float* t, int n, int batch,
                       int epochs, float lr, unsigned long long seed, float* epoch_loss,
                       void* stream) {
  if (!nin_supported(nin) || !params || !X || !t || n < 1 || batch < 1 || epochs < 0 || !(lr > 0.0f))
    return CR_E_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = param_count(nin);
  float *grad = nullptr, *mom = nullptr, *var = nullptr, *bl = nullptr, *el = nullptr, *part = nullptr;
  int* idx = nullptr;
  cr_status st = CR_OK;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && st == CR_OK) st = (e == cudaErrorMemoryAllocation) ? CR_E_NOMEM : CR_E_CUDA;
    return st == CR_OK;
  };
  ok(cudaMalloc(&grad, sizeof(float) * P));
  ok(cudaMalloc(&mom, sizeof(float) * P));
  ok(cudaMalloc(&var, sizeof(float) * P));
  ok(cudaMalloc(&bl, sizeof(float)));
  ok(cudaMalloc(&el, sizeof(float)));
  ok(cudaMalloc(&idx, sizeof(int) * n));
  ok(cudaMalloc(&part, sizeof(float) * (size_t)grad_blocks(batch < n ? batch : n) * (P + 1)));
  if (st == CR_OK) {
    ok(cudaMemsetAsync(mom, 0, sizeof(float) * P, s));
    ok(cudaMemsetAsync(var, 0, sizeof(float) * P, s));
  }
  std::vector<int> perm(n);
  uint64_t rs = seed;
  int step = 0;
  float last = 0.0f;
  for (int ep = 0; ep < epochs && st == CR_OK; ++ep) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) {  // Fisher-Yates with a seeded splitmix64
      const int j = int(splitmix64(&rs) % uint64_t(i + 1));
      const int tmp = perm[i];
      perm[i] = perm[j];
      perm[j] = tmp;
    }
    ok(cudaMemcpyAsync(idx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    ok(cudaMemsetAsync(el, 0, sizeof(float), s));
    int nb = 0;
    for (int b0 = 0; b0 < n && st == CR_OK; b0 += batch, ++nb) {
      const int cnt = b0 + batch <= n ? batch : n - b0;
      ok(dispatch_grad(nin, params, X, t, idx + b0, cnt, part, grad, bl, s));
      ++step;
      const float c1 = 1.0f - powf(0.9f, float(step)), c2 = 1.0f - powf(0.999f, float(step));
      k_mlp_adam<<<(P + 255) / 256, 256, 0, s>>>(params, grad, mom, var, P, lr, c1, c2);
      ok(cudaGetLastError());
      k_accumulate<<<1, 1, 0, s>>>(el, bl);
      ok(cudaGetLastError());
    }
    float sum = 0.0f;
    ok(cudaMemcpyAsync(&sum, el, sizeof(float), cudaMemcpyDeviceToHost, s));
    ok(cudaStreamSynchronize(s));
    last = nb > 0 ? sum / nb : 0.0f;
  }
  if (epoch_loss) *epoch_loss = last;
  cudaFree(grad);
  cudaFree(mom);
  cudaFree(var);
  cudaFree(bl);
  cudaFree(el);
  cudaFree(idx);
  cudaFree(part);
  return st;
}

}  // extern "C"
