// Training of the MLP Q-function (an extension: the paper uses tables and names deep RL
// as future work, Section 7): fitted-Q regression on transitions the solver generated.
//
// Network 16 -> H -> H -> 4 * nprec (ReLU), fp32, parameters in the layout
// W1[H][16], b1[H], W2[H][H], b2[H], W3[4 nprec][H], b3[4 nprec].
// Loss over a batch of B transitions: (1 / (4 B)) sum_b sum_j 1/2 (Q(f_b)[j, a_bj] - y_bj)^2
// with targets y_bj = r_b + gamma (1 - done_b) max_p Q_target(f'_b)[j, p] (or given targets).
//
// Each CTA takes a contiguous chunk of the batch and processes its samples one after the
// other: the whole CTA evaluates the layers (weights read through the read-only path,
// activations in shared memory), then every thread adds the gradient contributions of the
// parameters it owns (indices t, t + blockDim, ...) to a shared-memory accumulator. No
// atomics: the result is deterministic. A second kernel sums the CTA partials in CTA order
// and applies Adam (Kingma and Ba, ICLR 2015).
#include "internal.h"

namespace mpcg {

namespace {

constexpr int kMlpThreads = 256;
constexpr int kMaxOut = 32;

struct MlpShape {
  int H, nout, nprec;
  long long np;
  long long oW1, ob1, oW2, ob2, oW3, ob3;
};

__host__ __device__ MlpShape mlp_shape(int H, int nprec) {
  MlpShape s;
  s.H = H;
  s.nprec = nprec;
  s.nout = 4 * nprec;
  s.oW1 = 0;
  s.ob1 = s.oW1 + (long long)H * kNFeat;
  s.oW2 = s.ob1 + H;
  s.ob2 = s.oW2 + (long long)H * H;
  s.oW3 = s.ob2 + H;
  s.ob3 = s.oW3 + (long long)s.nout * H;
  s.np = s.ob3 + s.nout;
  return s;
}

// Forward pass of one sample by the whole CTA; f, h1, h2, out in shared memory.
__device__ void fwd(const float* __restrict__ w, const MlpShape& s, const float* f, float* h1, float* h2, float* out) {
  for (int i = threadIdx.x; i < s.H; i += blockDim.x) {
    float a = __ldg(w + s.ob1 + i);
    for (int j = 0; j < kNFeat; ++j) a = fmaf(__ldg(w + s.oW1 + i * kNFeat + j), f[j], a);
    h1[i] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s.H; i += blockDim.x) {
    float a = __ldg(w + s.ob2 + i);
    for (int j = 0; j < s.H; ++j) a = fmaf(__ldg(w + s.oW2 + (long long)i * s.H + j), h1[j], a);
    h2[i] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s.nout; i += blockDim.x) {
    float a = __ldg(w + s.ob3 + i);
    for (int j = 0; j < s.H; ++j) a = fmaf(__ldg(w + s.oW3 + (long long)i * s.H + j), h2[j], a);
    out[i] = a;
  }
  __syncthreads();
}

// r + gamma (1 - done) max over the entries p allowed for operation j of out[j nprec + p]
// (the one-step Bellman backup of Section 4.1 with Q given by the network).
__device__ __forceinline__ float target_of(const float* out, int nprec, int j, const OpMask& mask, float r, int done,
                                           float gamma) {
  float m = -INFINITY;
  for (int p = 0; p < nprec; ++p)
    if ((mask.m[j] >> p) & 1u) m = fmaxf(m, out[j * nprec + p]);
  return r + (done ? 0.f : gamma * m);
}

// Fitted-Q targets y[b][4] from the target network wt on feats_next[b], one CTA per sample.
__global__ void __launch_bounds__(kMlpThreads) mlp_targets_kernel(const float* __restrict__ wt, int H, int nprec,
                                                                  const float* __restrict__ feats_next,
                                                                  const float* __restrict__ rew,
                                                                  const int* __restrict__ done, int B, float gamma,
                                                                  OpMask mask, float* y) {
  extern __shared__ float sh[];
  const MlpShape s = mlp_shape(H, nprec);
  float* f = sh;
  float* h1 = f + kNFeat;
  float* h2 = h1 + s.H;
  float* out = h2 + s.H;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    if (threadIdx.x < kNFeat) f[threadIdx.x] = feats_next[(long long)b * kNFeat + threadIdx.x];
    __syncthreads();
    fwd(wt, s, f, h1, h2, out);
    if (threadIdx.x < 4) y[(long long)b * 4 + threadIdx.x] = target_of(out, nprec, threadIdx.x, mask, rew[b], done[b], gamma);
    __syncthreads();
  }
}

// One chunk of the batch per CTA: gradient partials of the CTA -> part[blockIdx.x][np],
// loss partial -> lpart[blockIdx.x]. With y == nullptr the targets come from the target
// network on the next features (fitted Q); otherwise y[b][4] are the targets.
__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(
    const float* __restrict__ w, const float* __restrict__ wt, int H, int nprec, const float* __restrict__ feats,
    const float* __restrict__ feats_next, const int* __restrict__ acts, const float* __restrict__ rew,
    const int* __restrict__ done, const float* __restrict__ y, const long long* __restrict__ idx, int B, int chunk,
    float gamma, OpMask mask, float* part, double* lpart) {
  extern __shared__ float sh[];
  const MlpShape s = mlp_shape(H, nprec);
  float* g = sh;                      // [np] gradient accumulator
  float* f = g + s.np;                // [16]
  float* h1 = f + kNFeat;             // [H]
  float* h2 = h1 + s.H;               // [H]
  float* out = h2 + s.H;              // [nout]
  float* dout = out + kMaxOut;        // [nout]
  float* dh2 = dout + kMaxOut;        // [H]
  float* dh1 = dh2 + s.H;             // [H]
  float* yt = dh1 + s.H;              // [4]
  __shared__ double lsum;
  for (long long i = threadIdx.x; i < s.np; i += blockDim.x) g[i] = 0.f;
  if (threadIdx.x == 0) lsum = 0.0;
  __syncthreads();
  const float scale = 1.f / (4.f * (float)B);
  const int b0 = blockIdx.x * chunk;
  const int b1 = min(B, b0 + chunk);
  for (int bi = b0; bi < b1; ++bi) {
    const long long src = idx ? idx[bi] : bi;
    // targets
    if (y) {
      if (threadIdx.x < 4) yt[threadIdx.x] = y[bi * 4 + threadIdx.x];
      __syncthreads();
    } else {
      if (threadIdx.x < kNFeat) f[threadIdx.x] = feats_next[src * kNFeat + threadIdx.x];
      __syncthreads();
      fwd(wt, s, f, h1, h2, out);
      if (threadIdx.x < 4) yt[threadIdx.x] = target_of(out, nprec, threadIdx.x, mask, rew[src], done[src], gamma);
      __syncthreads();
    }
    if (threadIdx.x < kNFeat) f[threadIdx.x] = feats[src * kNFeat + threadIdx.x];
    __syncthreads();
    fwd(w, s, f, h1, h2, out);
    // output error: only the taken action of each operation carries gradient
    for (int i = threadIdx.x; i < s.nout; i += blockDim.x) dout[i] = 0.f;
    __syncthreads();
    if (threadIdx.x == 0) {
      double l = 0.0;
      for (int j = 0; j < 4; ++j) {
        const int o = j * nprec + acts[src * 4 + j];
        const float d = out[o] - yt[j];
        dout[o] += d * scale;
        l += 0.5 * (double)d * (double)d;
      }
      lsum += l * (double)scale;
    }
    __syncthreads();
    // back through layer 3 and 2
    for (int k = threadIdx.x; k < s.H; k += blockDim.x) {
      float a = 0.f;
      for (int o = 0; o < s.nout; ++o) a = fmaf(__ldg(w + s.oW3 + (long long)o * s.H + k), dout[o], a);
      dh2[k] = h2[k] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < s.H; k += blockDim.x) {
      float a = 0.f;
      for (int i = 0; i < s.H; ++i) a = fmaf(__ldg(w + s.oW2 + (long long)i * s.H + k), dh2[i], a);
      dh1[k] = h1[k] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // parameter gradients, each thread on the indices it owns
    for (long long p = threadIdx.x; p < s.np; p += blockDim.x) {
      float d;
      if (p < s.ob1) d = dh1[p / kNFeat] * f[p % kNFeat];
      else if (p < s.oW2) d = dh1[p - s.ob1];
      else if (p < s.ob2) { const long long q = p - s.oW2; d = dh2[q / s.H] * h1[q % s.H]; }
      else if (p < s.oW3) d = dh2[p - s.ob2];
      else if (p < s.ob3) { const long long q = p - s.oW3; d = dout[q / s.H] * h2[q % s.H]; }
      else d = dout[p - s.ob3];
      g[p] += d;
    }
    __syncthreads();
  }
  float* dst = part + (long long)blockIdx.x * s.np;
  for (long long i = threadIdx.x; i < s.np; i += blockDim.x) dst[i] = g[i];
  if (threadIdx.x == 0) lpart[blockIdx.x] = lsum;
}

// Sums the CTA partials (CTA order) into grad; optionally applies Adam step t to w.
__global__ void mlp_reduce_adam_kernel(const float* __restrict__ part, int nparts, long long np, float* grad, float* w,
                                       float* m, float* v, int t, float lr, float b1, float b2, float eps,
                                       const double* lpart, double* loss) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
    float gi = 0.f;
    for (int c = 0; c < nparts; ++c) gi += part[(long long)c * np + i];
    if (grad) grad[i] = gi;
    if (w) {
      const float mi = b1 * m[i] + (1.f - b1) * gi;
      const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
      m[i] = mi;
      v[i] = vi;
      const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
      w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
  }
  if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
    double l = 0.0;
    for (int c = 0; c < nparts; ++c) l += lpart[c];
    *loss = l;
  }
}

// Minibatch indices for step t: Philox4x64-10 with key (seed, 0x6d6c7030) and counter
// (t, b, 0, 0), word 0 mod count.
__global__ void mlp_sample_kernel(long long* idx, int B, long long count, unsigned long long seed, unsigned long long t) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    U64x4 c;
    c.v[0] = t;
    c.v[1] = (unsigned long long)b;
    c.v[2] = 0;
    c.v[3] = 0;
    const U64x4 r = philox4x64_10(c, seed, 0x6d6c7030ull);
    idx[b] = (long long)(r.v[0] % (unsigned long long)count);
  }
}

}  // namespace

long long mlp_nparams_dev(int H, int nprec) { return mlp_shape(H, nprec).np; }

size_t mlp_grad_smem(int H, int nprec) {
  const MlpShape s = mlp_shape(H, nprec);
  return sizeof(float) * (size_t)(s.np + kNFeat + 4 * H + 2 * kMaxOut + 4);
}

cudaError_t mlp_set_smem_limit(size_t bytes) {
  return cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_mlp_grad(const float* w, const float* wt, int H, int nprec, const float* feats,
                            const float* feats_next, const int* acts, const float* rew, const int* done, const float* y,
                            const long long* idx, int B, int chunk, float gamma, OpMask mask, float* part,
                            double* lpart, cudaStream_t s) {
  const int nparts = (B + chunk - 1) / chunk;
  cudaGetLastError();
  mlp_grad_kernel<<<nparts, kMlpThreads, mlp_grad_smem(H, nprec), s>>>(w, wt, H, nprec, feats, feats_next, acts, rew,
                                                                       done, y, idx, B, chunk, gamma, mask, part, lpart);
  return cudaGetLastError();
}

cudaError_t launch_mlp_targets(const float* wt, int H, int nprec, const float* feats_next, const float* rew,
                               const int* done, int B, float gamma, OpMask mask, float* y, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const MlpShape sh = mlp_shape(H, nprec);
  const size_t smem = sizeof(float) * (size_t)(kNFeat + 2 * sh.H + sh.nout);
  cudaGetLastError();
  mlp_targets_kernel<<<B < 1024 ? B : 1024, kMlpThreads, smem, s>>>(wt, H, nprec, feats_next, rew, done, B, gamma,
                                                                     mask, y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_reduce_adam(const float* part, int nparts, long long np, float* grad, float* w, float* m,
                                   float* v, int t, float lr, const double* lpart, double* loss, cudaStream_t s) {
  cudaGetLastError();
  mlp_reduce_adam_kernel<<<(int)((np + 255) / 256), 256, 0, s>>>(part, nparts, np, grad, w, m, v, t, lr, 0.9f, 0.999f,
                                                                  1e-8f, lpart, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_sample(long long* idx, int B, long long count, unsigned long long seed, unsigned long long t,
                              cudaStream_t s) {
  cudaGetLastError();
  mlp_sample_kernel<<<(B + 255) / 256, 256, 0, s>>>(idx, B, count, seed, t);
  return cudaGetLastError();
}

}  // namespace mpcg
