// Learned con2prim guess: a 5 -> 64 -> 64 -> 1 tanh network with BF16
// operands and FP32 accumulation on the tensor cores (mma.sync m16n8k16),
// predicting log(mu) of the Kastaun et al. root from five features of the
// KRP variables.  Hand-written inference, forward + backward training step,
// Adam, and the bracket that the FP64 solve starts from.  The paper has no
// such network; the FP64 bracketed solve stays the refinement and decides the
// root.
#include <cuda_bf16.h>

#include "dev.cuh"
#include "internal.h"

namespace grmhd {

namespace {

__device__ __forceinline__ unsigned pack2(float lo, float hi) {
  __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}
__device__ __forceinline__ unsigned pack2b(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}
__device__ __forceinline__ void mma16816(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// A fragment (16x16) of an fp32 matrix, element (m,k) at A[m*sm + k*sk], origin (m0,k0)
__device__ __forceinline__ void frag_a(const float* A, int sm, int sk, int m0, int k0, unsigned* a) {
  const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
  const int r0 = m0 + g, r1 = r0 + 8, c0 = k0 + 2 * t, c1 = c0 + 8;
  a[0] = pack2(A[r0 * sm + c0 * sk], A[r0 * sm + (c0 + 1) * sk]);
  a[1] = pack2(A[r1 * sm + c0 * sk], A[r1 * sm + (c0 + 1) * sk]);
  a[2] = pack2(A[r0 * sm + c1 * sk], A[r0 * sm + (c1 + 1) * sk]);
  a[3] = pack2(A[r1 * sm + c1 * sk], A[r1 * sm + (c1 + 1) * sk]);
}
// B fragment (16x8) of an fp32 matrix, element (k,n) at B[k*sk + n*sn], origin (k0,n0)
__device__ __forceinline__ void frag_b(const float* B, int sk, int sn, int k0, int n0, unsigned* b) {
  const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
  const int n = n0 + g, k = k0 + 2 * t;
  b[0] = pack2(B[k * sk + n * sn], B[(k + 1) * sk + n * sn]);
  b[1] = pack2(B[(k + 8) * sk + n * sn], B[(k + 9) * sk + n * sn]);
}
// B fragment of a bf16 matrix
__device__ __forceinline__ void frag_bh(const __nv_bfloat16* B, int sk, int sn, int k0, int n0, unsigned* b) {
  const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
  const int n = n0 + g, k = k0 + 2 * t;
  b[0] = pack2b(B[k * sk + n * sn], B[(k + 1) * sk + n * sn]);
  b[1] = pack2b(B[(k + 8) * sk + n * sn], B[(k + 9) * sk + n * sn]);
}
// store a C fragment (16x8) to an fp32 matrix C[m*ld + n] at origin (m0,n0)
template <class F>
__device__ __forceinline__ void frag_c_apply(const float* c, int m0, int n0, F&& f) {
  const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
  f(m0 + g, n0 + 2 * t, c[0]);
  f(m0 + g, n0 + 2 * t + 1, c[1]);
  f(m0 + g + 8, n0 + 2 * t, c[2]);
  f(m0 + g + 8, n0 + 2 * t + 1, c[3]);
}

constexpr int NH = MLP_NH;
// per-warp shared buffers (floats) of the training step
constexpr int S_X = 0, S_H1 = 32 * 16, S_H2 = S_H1 + 32 * NH, S_DZ2 = S_H2 + 32 * NH, S_DZ1 = S_DZ2 + 32 * NH,
              S_Y = S_DZ1 + 32 * NH, S_T = S_Y + 32, S_WARP = S_T + 32;

// normalised features of the warp's 32 samples into Xs [32][16] (cols >= 5 zero)
__device__ __forceinline__ void load_x(float* Xs, const float* feat, long long idx, bool valid, const MlpNorm& nm) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int f = 0; f < 16; f++) {
    float v = 0.0f;
    if (valid && f < MLP_NIN) v = (feat[idx * MLP_FSTRIDE + f] - nm.fmean[f]) * nm.finv[f];
    Xs[lane * 16 + f] = v;
  }
}

// forward of 32 samples: H1, H2 (fp32) and y (normalised output) in smem;
// H2 may alias H1
__device__ __forceinline__ void warp_forward(const float* Xs, float* H1, float* H2, float* Y,
                                             const __nv_bfloat16* wb, const float* w) {
  __syncwarp();
  // layer 1: [32 x 16] x W1p^T, W1p [64][16] bf16
  for (int mt = 0; mt < 2; mt++) {
    unsigned a[4];
    frag_a(Xs, 16, 1, 16 * mt, 0, a);
    for (int nt = 0; nt < NH / 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      unsigned b[2];
      frag_bh(wb + MLP_BF_W1, 1, 16, 0, 8 * nt, b);
      mma16816(c, a, b);
      frag_c_apply(c, 16 * mt, 8 * nt, [&](int m, int n, float v) { H1[m * NH + n] = tanhf(v + w[MLP_B1 + n]); });
    }
  }
  __syncwarp();
  // layer 2: [32 x 64] x W2^T
  for (int mt = 0; mt < 2; mt++) {
    unsigned a[4][4];
    for (int kt = 0; kt < 4; kt++) frag_a(H1, NH, 1, 16 * mt, 16 * kt, a[kt]);
    __syncwarp();
    for (int nt = 0; nt < NH / 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      for (int kt = 0; kt < 4; kt++) {
        unsigned b[2];
        frag_bh(wb + MLP_BF_W2, 1, NH, 16 * kt, 8 * nt, b);
        mma16816(c, a[kt], b);
      }
      frag_c_apply(c, 16 * mt, 8 * nt, [&](int m, int n, float v) { H2[m * NH + n] = tanhf(v + w[MLP_B2 + n]); });
    }
  }
  __syncwarp();
  // layer 3: [32 x 64] x W3p^T, W3p [8][64] (row 0 = w3)
  for (int mt = 0; mt < 2; mt++) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kt = 0; kt < 4; kt++) {
      unsigned a[4], b[2];
      frag_a(H2, NH, 1, 16 * mt, 16 * kt, a);
      frag_bh(wb + MLP_BF_W3, 1, NH, 16 * kt, 0, b);
      mma16816(c, a, b);
    }
    frag_c_apply(c, 16 * mt, 0, [&](int m, int n, float v) {
      if (n == 0) Y[m] = v + w[MLP_B3];
    });
  }
  __syncwarp();
}

}  // namespace

// ------------------------------------------------------------------ inference
// Inference keeps every activation in registers.  With m16n8k16 fragments the
// accumulator of two neighbouring 8-column tiles of one layer holds, lane for
// lane, the A operand of the next layer's 16-column k-tile (rows g and g+8,
// columns 2t, 2t+1 and 2t+8, 2t+9 of lane (g, t)), so bias, activation and the
// bf16 packing turn one layer's output into the next layer's input without
// shared memory.  The activation is tanh.approx.bf16x2 on the packed pair; the
// output layer (64 -> 1) is a dot product over the lane's 16 columns reduced
// over the four lanes of a quad.  The weights sit in shared memory in fragment
// order ([fragment][lane] words), so every operand load is one conflict-free
// 32-bit load.
struct NetSmem {
  unsigned w1[8][2][32];      // B fragments of W1p [64][16]: [n-tile][reg][lane]
  unsigned w2[4][8][2][32];   // B fragments of W2: [k-tile][n-tile][reg][lane]
  float b1[8][2][32];         // b1 of the lane's two columns of each n-tile
  float b2[8][2][32];
  float w3[8][2][32];
  float b3, ymean, ystd, pad_;
  float fmean[MLP_NIN], finv[MLP_NIN];
};
constexpr size_t NET_XS_WORDS = 32 * 4;   // per warp: 32 rows of 8 bf16 inputs

__device__ __forceinline__ unsigned bf2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}
__device__ __forceinline__ unsigned tanh_bf2(unsigned x) {
  unsigned y;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}
__device__ __forceinline__ float bf_lo(unsigned x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf_hi(unsigned x) { return __uint_as_float(x & 0xffff0000u); }

// Fill the fragment-ordered operands (every thread of the CTA takes part).
__device__ void net_smem_fill(NetSmem& S, const __nv_bfloat16* __restrict__ wb, const float* __restrict__ w,
                              const MlpNorm& nm) {
  auto pk = [](__nv_bfloat16 a, __nv_bfloat16 b) {
    return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
  };
  for (int e = threadIdx.x; e < 8 * 2 * 32; e += blockDim.x) {
    const int lane = e & 31, r = (e >> 5) & 1, nt = e >> 6;
    const int g = lane >> 2, t = lane & 3, n = 8 * nt + g, k = 2 * t + 8 * r;
    // W1p [64][16]: B(k, n) = W1p[n][k]
    S.w1[nt][r][lane] = pk(wb[MLP_BF_W1 + n * 16 + k], wb[MLP_BF_W1 + n * 16 + k + 1]);
    const int c = 8 * nt + 2 * t + r;   // column of this lane's value r
    S.b1[nt][r][lane] = w[MLP_B1 + c];
    S.b2[nt][r][lane] = w[MLP_B2 + c];
    S.w3[nt][r][lane] = __bfloat162float(wb[MLP_BF_W3 + c]);
  }
  for (int e = threadIdx.x; e < 4 * 8 * 2 * 32; e += blockDim.x) {
    const int lane = e & 31, r = (e >> 5) & 1, nt = (e >> 6) & 7, kt = e >> 9;
    const int g = lane >> 2, t = lane & 3, n = 8 * nt + g, k = 16 * kt + 2 * t + 8 * r;
    // W2 [64][64] (out, in): B(k, n) = W2[n][k]
    S.w2[kt][nt][r][lane] = pk(wb[MLP_BF_W2 + n * MLP_NH + k], wb[MLP_BF_W2 + n * MLP_NH + k + 1]);
  }
  if (threadIdx.x == 0) {
    S.b3 = w[MLP_B3];
    S.ymean = nm.ymean;
    S.ystd = nm.ystd;
    for (int f = 0; f < MLP_NIN; f++) {
      S.fmean[f] = nm.fmean[f];
      S.finv[f] = nm.finv[f];
    }
  }
}

// The network on the warp's 32 samples: x[5] are the lane's raw features
// (zeros for an unused lane); returns the lane's de-normalised prediction.
// xs: this warp's NET_XS_WORDS words of shared memory.  Whole warp only.
__device__ __forceinline__ float net_warp(const NetSmem& S, unsigned* xs, const float* x) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float z[MLP_NIN];
#pragma unroll
  for (int f = 0; f < MLP_NIN; f++) z[f] = (x[f] - S.fmean[f]) * S.finv[f];
  __syncwarp();
  xs[4 * lane + 0] = bf2(z[0], z[1]);
  xs[4 * lane + 1] = bf2(z[2], z[3]);
  xs[4 * lane + 2] = bf2(z[4], 0.0f);
  xs[4 * lane + 3] = 0u;
  __syncwarp();
  float ymine = 0.0f;
#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
    // layer 1: A = inputs of rows 16 mt + g and 16 mt + g + 8 (k >= 8 zero)
    unsigned a[4] = {xs[4 * (16 * mt + g) + t], xs[4 * (16 * mt + g + 8) + t], 0u, 0u};
    unsigned h1[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const unsigned b[2] = {S.w1[nt][0][lane], S.w1[nt][1][lane]};
      mma16816(c, a, b);
      const float bl = S.b1[nt][0][lane], bh = S.b1[nt][1][lane];
      h1[nt >> 1][(nt & 1) * 2 + 0] = tanh_bf2(bf2(c[0] + bl, c[1] + bh));
      h1[nt >> 1][(nt & 1) * 2 + 1] = tanh_bf2(bf2(c[2] + bl, c[3] + bh));
    }
    // layer 2 and the output dot product
    float ylo = 0.0f, yhi = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kt = 0; kt < 4; kt++) {
        const unsigned b[2] = {S.w2[kt][nt][0][lane], S.w2[kt][nt][1][lane]};
        mma16816(c, h1[kt], b);
      }
      const float bl = S.b2[nt][0][lane], bh = S.b2[nt][1][lane];
      const float ul = S.w3[nt][0][lane], uh = S.w3[nt][1][lane];
      const unsigned r0 = tanh_bf2(bf2(c[0] + bl, c[1] + bh));
      const unsigned r1 = tanh_bf2(bf2(c[2] + bl, c[3] + bh));
      ylo = fmaf(ul, bf_lo(r0), fmaf(uh, bf_hi(r0), ylo));
      yhi = fmaf(ul, bf_lo(r1), fmaf(uh, bf_hi(r1), yhi));
    }
    ylo += __shfl_xor_sync(0xffffffffu, ylo, 1);
    ylo += __shfl_xor_sync(0xffffffffu, ylo, 2);
    yhi += __shfl_xor_sync(0xffffffffu, yhi, 1);
    yhi += __shfl_xor_sync(0xffffffffu, yhi, 2);
    // row r of this M-tile lives in quad (r & 7): the low half for r < 8
    const int r = lane & 15;
    const float vl = __shfl_sync(0xffffffffu, ylo, 4 * (r & 7));
    const float vh = __shfl_sync(0xffffffffu, yhi, 4 * (r & 7));
    if ((lane >> 4) == mt) ymine = r < 8 ? vl : vh;
  }
  return (ymine + S.b3) * S.ystd + S.ymean;
}

size_t net_smem_bytes(int threads) { return sizeof(NetSmem) + sizeof(unsigned) * NET_XS_WORDS * (threads / 32); }

// out[i] = predicted log(mu) for n samples of features [n][MLP_FSTRIDE]
__global__ void __launch_bounds__(256) k_mlp_infer(const float* __restrict__ feat, long long n, MlpNorm nm,
                                                  const __nv_bfloat16* __restrict__ wb, const float* __restrict__ w,
                                                  float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char net_raw[];
  NetSmem& S = *reinterpret_cast<NetSmem*>(net_raw);
  unsigned* xs = reinterpret_cast<unsigned*>(net_raw + sizeof(NetSmem)) + NET_XS_WORDS * (threadIdx.x >> 5);
  net_smem_fill(S, wb, w, nm);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
       base += nwarps * 32) {
    const long long idx = base + lane;
    float x[MLP_NIN];
#pragma unroll
    for (int f = 0; f < MLP_NIN; f++) x[f] = idx < n ? feat[idx * MLP_FSTRIDE + f] : 0.0f;
    const float y = net_warp(S, xs, x);
    if (idx < n) out[idx] = y;
  }
}

// ----------------------------------------------------------------- training
// One step over `batch` samples starting at `off` of the permutation
// i -> (pa*i + pb) mod n: forward, MSE loss, backward, gradients summed into
// grad (fp32, atomic) and the summed squared error into loss.
__global__ void __launch_bounds__(64) k_mlp_train_step(const float* __restrict__ feat, const float* __restrict__ target,
                                                      long long n, long long pa, long long pb, long long off,
                                                      int batch, MlpNorm nm, const __nv_bfloat16* __restrict__ wb,
                                                      const float* __restrict__ w, float* grad, float* loss) {
  extern __shared__ float smem[];
  __nv_bfloat16* swb = (__nv_bfloat16*)smem;
  float* sg = smem + (MLP_NBF + 1) / 2;
  float* sw0 = sg + MLP_NPARAM;
  for (int i = threadIdx.x; i < MLP_NBF; i += blockDim.x) swb[i] = wb[i];
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) sg[i] = 0.0f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sw = sw0 + warp * S_WARP;
  float* Xs = sw + S_X;
  float* H1 = sw + S_H1;
  float* H2 = sw + S_H2;
  float* DZ2 = sw + S_DZ2;
  float* DZ1 = sw + S_DZ1;
  float* Y = sw + S_Y;
  float* T = sw + S_T;
  const int s = (blockIdx.x * (blockDim.x >> 5) + warp) * 32 + lane;
  const bool valid = s < batch;
  long long idx = 0;
  if (valid) {
    unsigned long long ii = (unsigned long long)((off + s) % n);
    idx = (long long)(((unsigned long long)pa * ii + (unsigned long long)pb) % (unsigned long long)n);
  }
  load_x(Xs, feat, idx, valid, nm);
  T[lane] = valid ? (target[idx] - nm.ymean) / nm.ystd : 0.0f;
  warp_forward(Xs, H1, H2, Y, swb, w);
  // dL/dy of the mean squared error over the batch
  const float r = valid ? Y[lane] - T[lane] : 0.0f;
  const float dy = 2.0f * r / (float)batch;
  float sq = r * r;
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if (lane == 0) atomicAdd(loss, sq);
  Y[lane] = dy;
  __syncwarp();
  // dZ2 = dy w3 (1 - H2^2); b3, w3 gradients
  for (int j = 0; j < NH; j++) {
    const float h = H2[lane * NH + j];
    DZ2[lane * NH + j] = dy * w[MLP_W3 + j] * (1.0f - h * h);
  }
  {
    float d3 = dy;
    for (int o = 16; o > 0; o >>= 1) d3 += __shfl_xor_sync(0xffffffffu, d3, o);
    if (lane == 0) atomicAdd(&sg[MLP_B3], d3);
  }
  __syncwarp();
  for (int j = lane; j < NH; j += 32) {
    float a = 0.f, b2 = 0.f;
    for (int q = 0; q < 32; q++) {
      a += Y[q] * H2[q * NH + j];
      b2 += DZ2[q * NH + j];
    }
    atomicAdd(&sg[MLP_W3 + j], a);
    atomicAdd(&sg[MLP_B2 + j], b2);
  }
  // dW2[j][i] = sum_s DZ2[s][j] H1[s][i]   (M = j, N = i, K = s)
  for (int mt = 0; mt < 4; mt++)
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      for (int kt = 0; kt < 2; kt++) {
        unsigned a[4], b[2];
        frag_a(DZ2, 1, NH, 16 * mt, 16 * kt, a);
        frag_b(H1, NH, 1, 16 * kt, 8 * nt, b);
        mma16816(c, a, b);
      }
      frag_c_apply(c, 16 * mt, 8 * nt, [&](int m, int nn, float v) { atomicAdd(&sg[MLP_W2 + m * NH + nn], v); });
    }
  // dH1 = DZ2 W2 (M = s, N = i, K = j); dZ1 = dH1 (1 - H1^2)
  for (int mt = 0; mt < 2; mt++)
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      for (int kt = 0; kt < 4; kt++) {
        unsigned a[4], b[2];
        frag_a(DZ2, NH, 1, 16 * mt, 16 * kt, a);
        frag_bh(swb + MLP_BF_W2, NH, 1, 16 * kt, 8 * nt, b);
        mma16816(c, a, b);
      }
      frag_c_apply(c, 16 * mt, 8 * nt, [&](int m, int nn, float v) {
        const float h = H1[m * NH + nn];
        DZ1[m * NH + nn] = v * (1.0f - h * h);
      });
    }
  __syncwarp();
  for (int j = lane; j < NH; j += 32) {
    float b1 = 0.f;
    for (int q = 0; q < 32; q++) b1 += DZ1[q * NH + j];
    atomicAdd(&sg[MLP_B1 + j], b1);
  }
  // dW1[i][f] = sum_s DZ1[s][i] X[s][f]   (M = i, N = f (8), K = s)
  for (int mt = 0; mt < 4; mt++) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kt = 0; kt < 2; kt++) {
      unsigned a[4], b[2];
      frag_a(DZ1, 1, NH, 16 * mt, 16 * kt, a);
      frag_b(Xs, 16, 1, 16 * kt, 0, b);
      mma16816(c, a, b);
    }
    frag_c_apply(c, 16 * mt, 0, [&](int m, int f, float v) {
      if (f < MLP_NIN) atomicAdd(&sg[MLP_W1 + m * MLP_NIN + f], v);
    });
  }
  __syncthreads();
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) {
    const float v = sg[i];
    if (v != 0.0f) atomicAdd(&grad[i], v);
  }
}

// Adam on the fp32 master weights; refreshes the bf16 operand copies and
// clears the gradient for the next step.
__global__ void k_mlp_adam(float* w, float* m, float* v, float* grad, float lr, float b1, float b2, float eps,
                           float c1, float c2, __nv_bfloat16* wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_NPARAM) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    grad[i] = 0.0f;
  }
}

// bf16 operand copies: W1p [64][16] (zero padded), W2 [64][64], W3p [8][64]
__global__ void k_mlp_pack(const float* w, __nv_bfloat16* wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_NBF) {
    float v = 0.0f;
    if (i < MLP_BF_W2) {
      const int r = i / 16, c = i % 16;
      if (c < MLP_NIN) v = w[MLP_W1 + r * MLP_NIN + c];
    } else if (i < MLP_BF_W3) {
      v = w[MLP_W2 + (i - MLP_BF_W2)];
    } else {
      const int r = (i - MLP_BF_W3) / NH, c = (i - MLP_BF_W3) % NH;
      if (r == 0) v = w[MLP_W3 + c];
    }
    wb[i] = __float2bfloat16_rn(v);
  }
}

// sums and sums of squares of the features and the target (double atomics)
__global__ void k_mlp_stats(const float* __restrict__ feat, const float* __restrict__ target, long long n,
                            double* acc) {
  double s[12] = {0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    for (int f = 0; f < MLP_NIN; f++) {
      const double x = feat[i * MLP_FSTRIDE + f];
      s[f] += x;
      s[6 + f] += x * x;
    }
    const double t = target[i];
    s[5] += t;
    s[11] += t * t;
  }
  for (int k = 0; k < 12; k++) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], v);
  }
}

// ------------------------------------ network guess, FP32 search, FP64 polish
// Cells with status 4.  The network runs here, on features formed in
// registers from the cell's KRP variables; its guess mu_g and mu_g e^delta
// start at most 5 FP32 secant steps (krp_secant32, dev.cuh), and the FP64
// polish (krp_polish) takes the root or leaves a bracket for the refill solve.
// Warps take tiles of 32 consecutive cells (the network is a warp-wide
// product).
__global__ void __launch_bounds__(128) k_krp_seed(Par P, KrpBuf kb, float delta, const __nv_bfloat16* __restrict__ wb,
                                                  const float* __restrict__ wf, MlpNorm nm,
                                                  unsigned long long* stats) {
  extern __shared__ __align__(16) unsigned char net_raw[];
  NetSmem& S = *reinterpret_cast<NetSmem*>(net_raw);
  unsigned* xs = reinterpret_cast<unsigned*>(net_raw + sizeof(NetSmem)) + NET_XS_WORDS * (threadIdx.x >> 5);
  net_smem_fill(S, wb, wf, nm);
  __syncthreads();
  const long long n = kb.n;
  const int lane = threadIdx.x & 31;
  unsigned s_fb = 0, s_f32 = 0;
  bool any0 = false;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
       base += nwarps * 32) {
    const long long i = base + lane;
    const bool act = i < n && kb.st[i] == 4;
    const unsigned any = __ballot_sync(0xffffffffu, act);
    if (!any) continue;
    KS s;
    const double* w = kb.w;
    s.qh = s.r2 = s.b2 = s.rb2 = s.rperp2 = 0.0;
    s.D = 1.0;
    if (act) {
      s.qh = w[KW_QH * n + i]; s.r2 = w[KW_R2 * n + i]; s.b2 = w[KW_B2 * n + i];
      s.rb2 = w[KW_RB2 * n + i]; s.rperp2 = w[KW_RP2 * n + i];
      s.D = w[KW_D * n + i];
    }
    s.gam = P.gam; s.eps_min = P.eps_atm; s.vmax2 = P.vmax2;
    float x[MLP_FSTRIDE];
    krp_features(s, x);
    if (!act)
      for (int f = 0; f < MLP_NIN; f++) x[f] = S.fmean[f];
    const float lg = net_warp(S, xs, x);
    if (!act) continue;
    const KSf sf = ks_f32(s);
    float x0 = __expf(lg);
    if (!(x0 > 1e-30f)) x0 = 1e-30f;
    if (x0 > 1.0f) x0 = 1.0f;
    float x1 = fminf(x0 * __expf(delta), 1.0f);
    if (x1 == x0) x1 = x0 * (1.0f - 1e-3f);
    const float m32 = krp_secant32(sf, x0, x1, 5, s_f32);
    const float isl = krp_islope32(sf, m32, s_f32);
    double a = 0.0, b = 1.0, Ga = -1.0, Gb = 1.0, mu = 0.0;
    int its = 0;
    bool fb;
    const int r = krp_polish(s, P, f64_of(m32), f64_of(isl), a, b, Ga, Gb, mu, its, fb);
    s_fb += fb ? 1u : 0u;
    kb.w[KW_A * n + i] = a; kb.w[KW_B * n + i] = b;
    kb.w[KW_GA * n + i] = Ga; kb.w[KW_GB * n + i] = Gb;
    kb.w[KW_MU * n + i] = mu;
    kb.it[i] = its;
    kb.st[i] = (unsigned char)(r == 0 ? 0 : (r == 1 ? 1 : 2));
    any0 |= r == 0;
  }
  warp_mark_solve(kb, any0);
  warp_flush(&stats[7], s_fb);
  warp_flush(&stats[8], s_f32);
}

// log(mu) of solved cells (training targets); NaN where the solve failed
__global__ void k_mlp_logmu(KrpBuf kb, float* out) {
  const long long n = kb.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = kb.st[i] == 1 ? (float)log(kb.w[KW_MU * n + i]) : __int_as_float(0x7fc00000);
}

// ------------------------------------------------------------------ launchers
void launch_mlp_logmu(const KrpBuf& kb, float* out, cudaStream_t s, int nsm) {
  k_mlp_logmu<<<nsm * 4, 256, 0, s>>>(kb, out);
}
size_t mlp_infer_smem() { return net_smem_bytes(256); }
size_t mlp_train_smem() { return sizeof(float) * ((MLP_NBF + 1) / 2 + MLP_NPARAM + 2 * S_WARP); }

int mlp_setup_attrs() {
  cudaError_t e1 = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_infer_smem());
  cudaError_t e2 =
      cudaFuncSetAttribute(k_mlp_train_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_train_smem());
  cudaError_t e3 = cudaFuncSetAttribute(k_krp_seed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)net_smem_bytes(128));
  return (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess) ? 0 : -1;
}
void launch_mlp_infer(const float* feat, long long n, const MlpNorm& nm, const __nv_bfloat16* wb, const float* w,
                      float* out, cudaStream_t s, int nsm) {
  long long warps = (n + 31) / 32;
  long long blocks = (warps + 7) / 8;
  int grid = (int)(blocks < (long long)nsm * 2 ? blocks : (long long)nsm * 2);
  if (grid < 1) grid = 1;
  k_mlp_infer<<<grid, 256, mlp_infer_smem(), s>>>(feat, n, nm, wb, w, out);
}
void launch_mlp_train_step(const float* feat, const float* target, long long n, long long pa, long long pb,
                           long long off, int batch, const MlpNorm& nm, const __nv_bfloat16* wb, const float* w,
                           float* grad, float* loss, cudaStream_t s) {
  int grid = (batch + 63) / 64;
  k_mlp_train_step<<<grid, 64, mlp_train_smem(), s>>>(feat, target, n, pa, pb, off, batch, nm, wb, w, grad, loss);
}
void launch_mlp_adam(float* w, float* m, float* v, float* grad, float lr, int t, __nv_bfloat16* wb, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f / (1.0f - powf(b1, (float)t)), c2 = 1.0f / (1.0f - powf(b2, (float)t));
  k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(w, m, v, grad, lr, b1, b2, 1e-8f, c1, c2, wb);
  k_mlp_pack<<<(MLP_NBF + 255) / 256, 256, 0, s>>>(w, wb);
}
void launch_mlp_pack(const float* w, __nv_bfloat16* wb, cudaStream_t s) {
  k_mlp_pack<<<(MLP_NBF + 255) / 256, 256, 0, s>>>(w, wb);
}
void launch_mlp_stats(const float* feat, const float* target, long long n, double* acc, cudaStream_t s, int nsm) {
  k_mlp_stats<<<nsm * 4, 256, 0, s>>>(feat, target, n, acc);
}
void launch_krp_seed(const Par& P, const KrpBuf& kb, float delta, const __nv_bfloat16* wb, const float* w,
                     const MlpNorm& nm, unsigned long long* stats, cudaStream_t s, int grid) {
  k_krp_seed<<<grid, 128, net_smem_bytes(128), s>>>(P, kb, delta, wb, w, nm, stats);
}
int occ_seed_kernel() {
  int o = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_krp_seed, 128, net_smem_bytes(128));
  return o;
}

}  // namespace grmhd
