// Learned Krylov controller: a two-layer MLP (8 features -> 64 -> 64, ReLU, FP32) with two heads
// on the second hidden layer: the Krylov dimension y of a local exponential (linear) and the
// logit of the acceptance of the dimension the controller then uses, floor(y) clamped to
// [1, 126] (logistic: is the residual test at that dimension passed).  Features are known after
// the first Lanczos step.  Trained on the GPU with these kernels on the log of the method's own
// adaptive solves: head 1 and the trunk by mean-squared error, then head 2 alone (trunk frozen)
// by the logistic loss, both with Adam.  Parameter layout (MLP_NPARAM floats):
//   W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3, W4[64], b4.
#include "tdvp_internal.cuh"

namespace {

constexpr int NIN = MLP_NIN, NH = MLP_NH, NP = MLP_NPARAM;
constexpr int OW1 = 0, OB1 = OW1 + NIN * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
constexpr int OW4 = OB3 + 1, OB4 = OW4 + NH;
static_assert(OW4 == MLP_NPARAM_K && OB4 + 1 == MLP_NPARAM, "parameter layout");
constexpr int SB = 64;   // samples per block

// Per-block partial gradients (and loss in slot NP) over the samples [b*SB, (b+1)*SB) of the
// mini-batch rows idx0..idx0+B-1 of the log (row = 8 features then the final Krylov dimension).
// head 0: L = mean (y - k)^2 over trunk and head 1; head 1: L = mean logistic loss of
// sigma(a) against [k <= kp], kp = floor(y) clamped to [1, 126], over head 2 only.
__global__ void __launch_bounds__(NH) mlp_grad_kernel(int head, const float* __restrict__ data, long long idx0,
                                                       int B, const float* __restrict__ w,
                                                       float* __restrict__ partial) {
  __shared__ float W2s[NH][NH + 1];
  __shared__ float x[NIN], h1[NH], h2[NH], dz2[NH], red[NH], red2[NH];
  const int j = threadIdx.x;
  for (int i = 0; i < NH; ++i) W2s[i][j] = w[OW2 + i * NH + j];
  float w1[NIN];
  for (int i = 0; i < NIN; ++i) w1[i] = w[OW1 + i * NH + j];
  const float b1 = w[OB1 + j], b2 = w[OB2 + j], w3 = w[OW3 + j], b3 = w[OB3], w4 = w[OW4 + j], b4 = w[OB4];
  float gW1[NIN] = {0}, gb1 = 0, gW2[NH], gb2 = 0, gW3 = 0, gb3 = 0, gW4 = 0, gb4 = 0, loss = 0;
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
    red2[j] = h2[j] * w4;
    __syncthreads();
    for (int o = NH / 2; o > 0; o >>= 1) {
      if (j < o) { red[j] += red[j + o]; red2[j] += red2[j + o]; }
      __syncthreads();
    }
    const float y = red[0] + b3;
    if (head == 1) {
      // acceptance of kp: label 1 if the solve's final dimension k <= kp
      const float kp = fminf(fmaxf(floorf(y), 1.f), 126.f);
      const float lab = t <= kp ? 1.f : 0.f;
      const float a = red2[0] + b4;
      const float p = 1.f / (1.f + expf(-a));
      const float da = (p - lab) / (float)B;
      // logistic loss log(1 + e^a) - lab * a, written without overflow
      if (j == 0) { gb4 += da; loss += (fmaxf(a, 0.f) + log1pf(expf(-fabsf(a))) - lab * a) / (float)B; }
      gW4 = fmaf(da, h2[j], gW4);
      __syncthreads();
      continue;
    }
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
  P[OW4 + j] = gW4;
  if (j == 0) { P[OB3] = gb3; P[OB4] = gb4; P[NP] = loss; }
}

// grad[p] = sum_b partial[b][p] in block order (deterministic); the loss (slot NP) is also added
// to *loss_acc, one launch after another in stream order
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int nblk, float* __restrict__ grad,
                                  float* __restrict__ loss_acc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NP) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += partial[(long long)b * (NP + 1) + p];
  grad[p] = s;
  if (p == NP && loss_acc) *loss_acc += s;
}

// Adam on params [p0, p1); the others keep their values
__global__ void mlp_adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, float lr, float c1, float c2, int p0, int p1) {
  const int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= p1) return;
  const float gp = g[p];
  const float mp = 0.9f * m[p] + 0.1f * gp;
  const float vp = 0.999f * v[p] + 0.001f * gp * gp;
  m[p] = mp;
  v[p] = vp;
  w[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + 1e-8f);
}

}  // namespace

int mlp_partial_floats(int B) { return ((B + SB - 1) / SB) * (NP + 1); }

cudaError_t launch_mlp_grad(int head, const float* data, long long idx0, int B, const float* w, float* partial,
                            float* grad, float* loss_acc, cudaStream_t st) {
  const int nblk = (B + SB - 1) / SB;
  mlp_grad_kernel<<<nblk, NH, 0, st>>>(head, data, idx0, B, w, partial);
  mlp_reduce_kernel<<<(NP + 1 + 255) / 256, 256, 0, st>>>(partial, nblk, grad, loss_acc);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* w, const float* g, float* m, float* v, float lr, int t, int p0, int p1,
                            cudaStream_t st) {
  const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
  mlp_adam_kernel<<<(p1 - p0 + 255) / 256, 256, 0, st>>>(w, g, m, v, lr, c1, c2, p0, p1);
  return cudaGetLastError();
}
