// Learned Krylov controller: a two-layer MLP (8 features -> 64 -> 64 -> 1, ReLU, FP32) that
// predicts the Krylov dimension of a local exponential from quantities known after its first
// Lanczos step.  Trained on the GPU with these kernels on the log of the method's own adaptive
// solves (mean-squared error, Adam).  Parameter layout (MLP_NPARAM floats):
//   W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3.
#include "tdvp_internal.cuh"

namespace {

constexpr int NIN = MLP_NIN, NH = MLP_NH, NP = MLP_NPARAM;
constexpr int OW1 = 0, OB1 = OW1 + NIN * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
constexpr int SB = 64;   // samples per block

// Per-block partial gradients (and loss in slot NP) over the samples [b*SB, (b+1)*SB) of the
// mini-batch rows idx0..idx0+B-1 of the log (row = 8 features then the target).
__global__ void __launch_bounds__(NH) mlp_grad_kernel(const float* __restrict__ data, long long idx0, int B,
                                                       const float* __restrict__ w, float* __restrict__ partial) {
  __shared__ float W2s[NH][NH + 1];
  __shared__ float x[NIN], h1[NH], h2[NH], dz2[NH], red[NH];
  const int j = threadIdx.x;
  for (int i = 0; i < NH; ++i) W2s[i][j] = w[OW2 + i * NH + j];
  float w1[NIN];
  for (int i = 0; i < NIN; ++i) w1[i] = w[OW1 + i * NH + j];
  const float b1 = w[OB1 + j], b2 = w[OB2 + j], w3 = w[OW3 + j], b3 = w[OB3];
  float gW1[NIN] = {0}, gb1 = 0, gW2[NH], gb2 = 0, gW3 = 0, gb3 = 0, loss = 0;
  for (int i = 0; i < NH; ++i) gW2[i] = 0;
  __syncthreads();
  const int s0 = blockIdx.x * SB, s1 = min(B, s0 + SB);
  for (int s = s0; s < s1; ++s) {
    const float* row = data + (idx0 + s) * (NIN + 1);
    if (j < NIN) x[j] = row[j];
    const float t = row[NIN];
    __syncthreads();
    float z1 = b1;
    for (int i = 0; i < NIN; ++i) z1 = fmaf(x[i], w1[i], z1);
    h1[j] = fmaxf(z1, 0.f);
    __syncthreads();
    float z2 = b2;
    for (int i = 0; i < NH; ++i) z2 = fmaf(h1[i], W2s[i][j], z2);
    h2[j] = fmaxf(z2, 0.f);
    red[j] = h2[j] * w3;
    __syncthreads();
    for (int o = NH / 2; o > 0; o >>= 1) {
      if (j < o) red[j] += red[j + o];
      __syncthreads();
    }
    const float y = red[0] + b3;
    const float r = y - t;
    const float dy = 2.f * r / (float)B;
    if (j == 0) { gb3 += dy; loss += r * r / (float)B; }
    gW3 = fmaf(dy, h2[j], gW3);
    dz2[j] = z2 > 0.f ? dy * w3 : 0.f;
    __syncthreads();
    const float dz2j = dz2[j];
    for (int i = 0; i < NH; ++i) gW2[i] = fmaf(h1[i], dz2j, gW2[i]);
    gb2 += dz2j;
    float dh1 = 0.f;
    for (int k = 0; k < NH; ++k) dh1 = fmaf(dz2[k], W2s[j][k], dh1);
    const float dz1 = z1 > 0.f ? dh1 : 0.f;
    for (int i = 0; i < NIN; ++i) gW1[i] = fmaf(x[i], dz1, gW1[i]);
    gb1 += dz1;
    __syncthreads();
  }
  float* P = partial + (long long)blockIdx.x * (NP + 1);
  for (int i = 0; i < NIN; ++i) P[OW1 + i * NH + j] = gW1[i];
  P[OB1 + j] = gb1;
  for (int i = 0; i < NH; ++i) P[OW2 + i * NH + j] = gW2[i];
  P[OB2 + j] = gb2;
  P[OW3 + j] = gW3;
  if (j == 0) { P[OB3] = gb3; P[NP] = loss; }
}

// grad[p] = sum_b partial[b][p] in block order (deterministic)
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int nblk, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NP) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += partial[(long long)b * (NP + 1) + p];
  grad[p] = s;
}

__global__ void mlp_adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NP) return;
  const float gp = g[p];
  const float mp = 0.9f * m[p] + 0.1f * gp;
  const float vp = 0.999f * v[p] + 0.001f * gp * gp;
  m[p] = mp;
  v[p] = vp;
  w[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + 1e-8f);
}

}  // namespace

int mlp_partial_floats(int B) { return ((B + SB - 1) / SB) * (NP + 1); }

cudaError_t launch_mlp_grad(const float* data, long long idx0, int B, const float* w, float* partial, float* grad,
                            cudaStream_t st) {
  const int nblk = (B + SB - 1) / SB;
  mlp_grad_kernel<<<nblk, NH, 0, st>>>(data, idx0, B, w, partial);
  mlp_reduce_kernel<<<(NP + 1 + 255) / 256, 256, 0, st>>>(partial, nblk, grad);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* w, const float* g, float* m, float* v, float lr, int t, cudaStream_t st) {
  const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
  mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, st>>>(w, g, m, v, lr, c1, c2);
  return cudaGetLastError();
}
