// Dynamic-aperture surrogate network: MLP 16 -> 256 -> 256 -> 256 -> 256 -> 2
// (exact GELU), BF16 weights and activations, FP32 accumulation on the tensor
// cores, FP32 master weights with Adam.  Hand-written forward, backward and
// optimiser kernels.
//
// Rounding points (the oracle rounds at the same places): the network input,
// every weight matrix, every hidden activation and every back-propagated
// pre-activation gradient dZ are bfloat16; accumulations, biases, GELU and its
// derivative, the head (256 -> 2), the loss and Adam are FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "xt_internal.h"
#include "xtgb.h"

namespace {

thread_local std::string g_err;
int fail(int code, const std::string& m) {
  g_err = m;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return XT_ERR_CUDA;
}
#define CK(call)                                        \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

typedef uint16_t bf16_t;  // storage type; converted with the cuda_bf16 intrinsics

constexpr int NL = 5;
constexpr int WIDTH[NL + 1] = {16, 256, 256, 256, 256, 2};
constexpr int64_t OFF_W[NL] = {0, 4352, 70144, 135936, 201728};
constexpr int64_t OFF_B[NL] = {4096, 69888, 135680, 201472, 202240};
constexpr int64_t NPARAM = XS_N_PARAMS;
static_assert(202242 == XS_N_PARAMS, "parameter count");

__device__ __forceinline__ float bf2f(bf16_t v) {
  return __bfloat162float(__ushort_as_bfloat16(v));
}
__device__ __forceinline__ bf16_t f2bf(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------------------
// C[M x N] = A[M x K] * B[N x K]^T with A, B bfloat16 (K contiguous), FP32
// accumulation on the tensor cores (mma.sync m16n8k16), K a multiple of 16.
// Block tile 64 x 64, 4 warps of 32 x 32.
enum { EPI_GELU = 0, EPI_DGRAD = 1, EPI_F32 = 2 };
struct Epi {
  const float* bias;    // EPI_GELU
  float* z;             // EPI_GELU: pre-activation out (may be null); EPI_DGRAD: fp32 dZ out
  const float* zprev;   // EPI_DGRAD: pre-activation of this layer's output
  bf16_t* out_b;        // EPI_GELU: activation; EPI_DGRAD: bf16 dZ
  float* out_f;         // EPI_F32
  int ld;               // leading dimension of every output / zprev
};

constexpr int TM = 64, TN = 64, TK = 16, SP = TK + 8;

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int EPI>
__global__ void __launch_bounds__(128) gemm_nt_kernel(const bf16_t* __restrict__ A, int lda,
                                                      const bf16_t* __restrict__ B, int ldb, int M, int N,
                                                      int K, Epi e) {
  __shared__ __align__(16) bf16_t As[TM][SP];
  __shared__ __align__(16) bf16_t Bs[TN][SP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;
  const int lr = tid >> 1, lc = (tid & 1) * 8;  // 64 rows x 2 halves of 8
  for (int k0 = 0; k0 < K; k0 += TK) {
    uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
    if (m0 + lr < M) va = *(const uint4*)(A + (int64_t)(m0 + lr) * lda + k0 + lc);
    if (n0 + lr < N) vb = *(const uint4*)(B + (int64_t)(n0 + lr) * ldb + k0 + lc);
    *(uint4*)&As[lr][lc] = va;
    *(uint4*)&Bs[lr][lc] = vb;
    __syncthreads();
    uint32_t af[2][4], bfr[4][2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int r = wm * 32 + i * 16 + g;
      af[i][0] = *(const uint32_t*)&As[r][2 * t];
      af[i][1] = *(const uint32_t*)&As[r + 8][2 * t];
      af[i][2] = *(const uint32_t*)&As[r][2 * t + 8];
      af[i][3] = *(const uint32_t*)&As[r + 8][2 * t + 8];
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int c = wn * 32 + j * 8 + g;
      bfr[j][0] = *(const uint32_t*)&Bs[c][2 * t];
      bfr[j][1] = *(const uint32_t*)&Bs[c][2 * t + 8];
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], af[i], bfr[j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; i++) {
#pragma unroll
    for (int j = 0; j < 4; j++) {
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int row = m0 + wm * 32 + i * 16 + g + ((q & 2) ? 8 : 0);
        const int col = n0 + wn * 32 + j * 8 + 2 * t + (q & 1);
        if (row >= M || col >= N) continue;
        const int64_t o = (int64_t)row * e.ld + col;
        const float v = acc[i][j][q];
        if (EPI == EPI_GELU) {
          const float z = v + e.bias[col];
          if (e.z) e.z[o] = z;
          e.out_b[o] = f2bf(gelu_f(z));
        } else if (EPI == EPI_DGRAD) {
          const float dz = v * gelu_grad_f(e.zprev[o]);
          e.z[o] = dz;
          e.out_b[o] = f2bf(dz);
        } else {
          e.out_f[o] = v;
        }
      }
    }
  }
}

template <int EPI>
int gemm(const bf16_t* A, int lda, const bf16_t* B, int ldb, int M, int N, int K, const Epi& e,
         cudaStream_t s) {
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_nt_kernel<EPI><<<grid, 128, 0, s>>>(A, lda, B, ldb, M, N, K, e);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void to_bf16_kernel(const float* __restrict__ x, bf16_t* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = f2bf(x[i]);
}

// bf16 copies of the weights: W (out x in) and W^T (in x out).
__global__ void refresh_weights_kernel(const float* __restrict__ master, bf16_t* __restrict__ wb,
                                       bf16_t* __restrict__ wtb, int out, int in) {
  const int64_t n = (int64_t)out * in;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / in), c = (int)(i % in);
    const bf16_t v = f2bf(master[i]);
    wb[i] = v;
    wtb[(int64_t)c * out + r] = v;
  }
}

// Head: out[b][j] = sum_k a4[b][k] W5[j][k] + b5[j], one warp per sample.
__global__ void head_forward_kernel(const bf16_t* __restrict__ a4, const bf16_t* __restrict__ w5,
                                    const float* __restrict__ b5, float* __restrict__ out, int64_t B) {
  const int lane = threadIdx.x & 31;
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= B) return;
  float s0 = 0.f, s1 = 0.f;
  for (int k = lane; k < 256; k += 32) {
    const float a = bf2f(a4[b * 256 + k]);
    s0 = fmaf(a, bf2f(w5[k]), s0);
    s1 = fmaf(a, bf2f(w5[256 + k]), s1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (lane == 0) {
    out[2 * b] = s0 + b5[0];
    out[2 * b + 1] = s1 + b5[1];
  }
}

__global__ void mask_count_kernel(const float* __restrict__ mask, int64_t B, float* __restrict__ cnt) {
  float s = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x)
    s += mask[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(cnt, s);
}

// Loss terms and dL/dout.  scal[0] += loss, scal[1] = sum(mask).
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ y,
                            const float* __restrict__ t, const float* __restrict__ mask, int64_t B, float lam,
                            float* __restrict__ dout, float* __restrict__ scal) {
  const float nm = fmaxf(scal[1], 1.0f);
  float s = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
    const float l = out[2 * i], p = out[2 * i + 1];
    const float bce = fmaxf(l, 0.f) - l * y[i] + log1pf(expf(-fabsf(l)));
    const float res = (p - t[i]) * mask[i];
    s += bce / (float)B + lam * res * res / nm;
    dout[2 * i] = (1.0f / (1.0f + expf(-l)) - y[i]) / (float)B;
    dout[2 * i + 1] = lam * 2.0f * res / nm;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&scal[0], s);
}

// Head backward: dW5, db5 (atomics over batch slices) and dZ4.
__global__ void head_backward_kernel(const float* __restrict__ dout, const bf16_t* __restrict__ a4,
                                     const bf16_t* __restrict__ w5, const float* __restrict__ z4, int64_t B,
                                     float* __restrict__ gw5, float* __restrict__ gb5, float* __restrict__ dzf,
                                     bf16_t* __restrict__ dzb) {
  const int k = threadIdx.x;  // 256 threads: one hidden unit each
  const float w0 = bf2f(w5[k]), w1 = bf2f(w5[256 + k]);
  float s0 = 0.f, s1 = 0.f, d0 = 0.f, d1 = 0.f;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    const float g0 = dout[2 * b], g1 = dout[2 * b + 1];
    const float a = bf2f(a4[b * 256 + k]);
    s0 = fmaf(g0, a, s0);
    s1 = fmaf(g1, a, s1);
    if (k == 0) { d0 += g0; d1 += g1; }
    const float dz = (g0 * w0 + g1 * w1) * gelu_grad_f(z4[b * 256 + k]);
    dzf[b * 256 + k] = dz;
    dzb[b * 256 + k] = f2bf(dz);
  }
  atomicAdd(&gw5[k], s0);
  atomicAdd(&gw5[256 + k], s1);
  if (k == 0) {
    atomicAdd(&gb5[0], d0);
    atomicAdd(&gb5[1], d1);
  }
}

// dst[c][b] = src[b][c] (bf16), rows b >= B of dst padded with zeros up to Bp.
__global__ void transpose_kernel(const bf16_t* __restrict__ src, int64_t B, int C, bf16_t* __restrict__ dst,
                                 int64_t Bp) {
  __shared__ bf16_t tile[32][33];
  const int64_t b0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t b = b0 + r;
    const int c = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (b < B && c < C) ? src[b * C + c] : (bf16_t)0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int c = c0 + r;
    const int64_t b = b0 + threadIdx.x;
    if (c < C && b < Bp) dst[(int64_t)c * Bp + b] = tile[threadIdx.x][r];
  }
}

// db[n] = sum_b dz[b][n]
__global__ void colsum_kernel(const float* __restrict__ dz, int64_t B, int C, float* __restrict__ db) {
  const int c = threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) s += dz[b * C + c];
  atomicAdd(&db[c], s);
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float c1, float c2,
                            float eps) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int grid_1d(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
struct xs_mlp {
  float* master = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  bf16_t* wb = nullptr;   // all layers' bf16 W, same offsets as the flat layout
  bf16_t* wtb = nullptr;  // all layers' bf16 W^T
  float* scal = nullptr;  // [0] loss [1] mask count
  int64_t step = 0;
  int64_t cap = 0;
  bf16_t* a[NL] = {nullptr};  // a0 .. a4
  float* z[NL - 1] = {nullptr};
  float* out = nullptr;
  float* dout = nullptr;
  float* dzf[2] = {nullptr};
  bf16_t* dzb[2] = {nullptr};
  bf16_t* dzT = nullptr;
  bf16_t* aT = nullptr;
};

static void free_ws(xs_mlp* n) {
  for (int i = 0; i < NL; i++) { cudaFree(n->a[i]); n->a[i] = nullptr; }
  for (int i = 0; i < NL - 1; i++) { cudaFree(n->z[i]); n->z[i] = nullptr; }
  for (int i = 0; i < 2; i++) { cudaFree(n->dzf[i]); cudaFree(n->dzb[i]); n->dzf[i] = nullptr; n->dzb[i] = nullptr; }
  cudaFree(n->out); cudaFree(n->dout); cudaFree(n->dzT); cudaFree(n->aT);
  n->out = n->dout = nullptr;
  n->dzT = n->aT = nullptr;
  n->cap = 0;
}

static int64_t pad16(int64_t b) { return (b + 15) / 16 * 16; }

static int ensure_ws(xs_mlp* n, int64_t B) {
  if (B <= n->cap) return XT_OK;
  free_ws(n);
  const int64_t C = 256, Bp = pad16(B);
  CK(cudaMalloc(&n->a[0], (size_t)Bp * 16 * sizeof(bf16_t)));
  for (int i = 1; i < NL; i++) CK(cudaMalloc(&n->a[i], (size_t)Bp * C * sizeof(bf16_t)));
  for (int i = 0; i < NL - 1; i++) CK(cudaMalloc(&n->z[i], (size_t)Bp * C * sizeof(float)));
  for (int i = 0; i < 2; i++) {
    CK(cudaMalloc(&n->dzf[i], (size_t)Bp * C * sizeof(float)));
    CK(cudaMalloc(&n->dzb[i], (size_t)Bp * C * sizeof(bf16_t)));
  }
  CK(cudaMalloc(&n->out, (size_t)Bp * 2 * sizeof(float)));
  CK(cudaMalloc(&n->dout, (size_t)Bp * 2 * sizeof(float)));
  CK(cudaMalloc(&n->dzT, (size_t)Bp * C * sizeof(bf16_t)));
  CK(cudaMalloc(&n->aT, (size_t)Bp * C * sizeof(bf16_t)));
  n->cap = B;
  return XT_OK;
}

static int refresh(xs_mlp* n, cudaStream_t s) {
  for (int l = 0; l < NL; l++) {
    const int out = WIDTH[l + 1], in = WIDTH[l];
    refresh_weights_kernel<<<grid_1d((int64_t)out * in, 256), 256, 0, s>>>(n->master + OFF_W[l], n->wb + OFF_W[l],
                                                                           n->wtb + OFF_W[l], out, in);
  }
  CK(cudaGetLastError());
  return XT_OK;
}

// Forward of the 4 hidden layers and the head on a batch already in a[0].
static int forward_layers(xs_mlp* n, int64_t B, bool keep_z, bf16_t** acts, float* out, cudaStream_t s) {
  for (int l = 0; l < NL - 1; l++) {
    Epi e;
    std::memset(&e, 0, sizeof(e));
    e.bias = n->master + OFF_B[l];
    e.z = keep_z ? n->z[l] : nullptr;
    e.out_b = acts[l + 1];
    e.ld = 256;
    int rc = gemm<EPI_GELU>(acts[l], WIDTH[l], n->wb + OFF_W[l], WIDTH[l], (int)B, 256, WIDTH[l], e, s);
    if (rc) return cuda_fail((cudaError_t)rc, "forward gemm");
  }
  const int64_t threads = B * 32;
  head_forward_kernel<<<(int)((threads + 255) / 256), 256, 0, s>>>(acts[NL - 1], n->wb + OFF_W[NL - 1],
                                                                 n->master + OFF_B[NL - 1], out, B);
  CK(cudaGetLastError());
  return XT_OK;
}

static int loss_grad(xs_mlp* n, const float* X, const float* y, const float* t, const float* mask, int64_t B,
                     float lam, cudaStream_t s) {
  int rc = ensure_ws(n, B);
  if (rc) return rc;
  to_bf16_kernel<<<grid_1d(B * 16, 256), 256, 0, s>>>(X, n->a[0], B * 16);
  CK(cudaGetLastError());
  rc = forward_layers(n, B, true, n->a, n->out, s);
  if (rc) return rc;
  CK(cudaMemsetAsync(n->scal, 0, 2 * sizeof(float), s));
  mask_count_kernel<<<grid_1d(B, 256), 256, 0, s>>>(mask, B, n->scal + 1);
  loss_kernel<<<grid_1d(B, 256), 256, 0, s>>>(n->out, y, t, mask, B, lam, n->dout, n->scal);
  CK(cudaMemsetAsync(n->grad, 0, NPARAM * sizeof(float), s));
  const int hb = (int)std::min<int64_t>(B, 1024);
  head_backward_kernel<<<hb, 256, 0, s>>>(n->dout, n->a[NL - 1], n->wb + OFF_W[NL - 1], n->z[NL - 2], B,
                                          n->grad + OFF_W[NL - 1], n->grad + OFF_B[NL - 1], n->dzf[0], n->dzb[0]);
  CK(cudaGetLastError());
  const int64_t Bp = pad16(B);
  int cur = 0;
  for (int l = NL - 2; l >= 0; l--) {
    const int in = WIDTH[l];
    // wgrad: dW_l = dZ^T a_{l}  (M = 256 outputs, N = in, K = batch)
    dim3 tb(32, 8);
    transpose_kernel<<<dim3((unsigned)((Bp + 31) / 32), 256 / 32), tb, 0, s>>>(n->dzb[cur], B, 256, n->dzT, Bp);
    transpose_kernel<<<dim3((unsigned)((Bp + 31) / 32), (in + 31) / 32), tb, 0, s>>>(n->a[l], B, in, n->aT, Bp);
    CK(cudaGetLastError());
    Epi e;
    std::memset(&e, 0, sizeof(e));
    e.out_f = n->grad + OFF_W[l];
    e.ld = in;
    rc = gemm<EPI_F32>(n->dzT, (int)Bp, n->aT, (int)Bp, 256, in, (int)Bp, e, s);
    if (rc) return cuda_fail((cudaError_t)rc, "wgrad gemm");
    colsum_kernel<<<(int)std::min<int64_t>(B, 1024), 256, 0, s>>>(n->dzf[cur], B, 256, n->grad + OFF_B[l]);
    CK(cudaGetLastError());
    if (l > 0) {
      // dgrad: dA_{l-1} = dZ_l W_l, then times GELU'(z_{l-1})
      Epi d;
      std::memset(&d, 0, sizeof(d));
      d.zprev = n->z[l - 1];
      d.z = n->dzf[1 - cur];
      d.out_b = n->dzb[1 - cur];
      d.ld = 256;
      rc = gemm<EPI_DGRAD>(n->dzb[cur], 256, n->wtb + OFF_W[l], 256, (int)B, 256, 256, d, s);
      if (rc) return cuda_fail((cudaError_t)rc, "dgrad gemm");
      cur = 1 - cur;
    }
  }
  return XT_OK;
}

extern "C" {

int xs_mlp_create(uint64_t seed, xs_mlp** out) {
  g_err.clear();
  if (!out) return fail(XT_ERR_INVALID, "out is null");
  *out = nullptr;
  xs_mlp* n = new xs_mlp();
  auto bail = [&](int rc) {
    xs_mlp_destroy(n);
    return rc;
  };
  if (cudaMalloc(&n->master, NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->m, NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->v, NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->grad, NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->wb, NPARAM * sizeof(bf16_t)) != cudaSuccess ||
      cudaMalloc(&n->wtb, NPARAM * sizeof(bf16_t)) != cudaSuccess ||
      cudaMalloc(&n->scal, 4 * sizeof(float)) != cudaSuccess)
    return bail(fail(XT_ERR_NOMEM, "cudaMalloc of the network parameters failed"));
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation on the host
  std::vector<float> h(NPARAM);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < NL; l++) {
    std::uniform_real_distribution<float> U(-1.0f / std::sqrt((float)WIDTH[l]), 1.0f / std::sqrt((float)WIDTH[l]));
    for (int64_t i = OFF_W[l]; i < OFF_W[l] + (int64_t)WIDTH[l + 1] * WIDTH[l]; i++) h[i] = U(rng);
    for (int64_t i = OFF_B[l]; i < OFF_B[l] + WIDTH[l + 1]; i++) h[i] = U(rng);
  }
  int rc = xs_mlp_set_params(n, h.data(), NPARAM, nullptr);
  if (rc) return bail(rc);
  *out = n;
  return XT_OK;
}

void xs_mlp_destroy(xs_mlp* n) {
  if (!n) return;
  cudaDeviceSynchronize();
  free_ws(n);
  cudaFree(n->master); cudaFree(n->m); cudaFree(n->v); cudaFree(n->grad);
  cudaFree(n->wb); cudaFree(n->wtb); cudaFree(n->scal);
  delete n;
}

int xs_mlp_set_params(xs_mlp* n, const float* params, int64_t count, void* stream) {
  g_err.clear();
  if (!n || !params || count != NPARAM) return fail(XT_ERR_INVALID, "need 202242 parameters");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(n->master, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(n->m, 0, NPARAM * sizeof(float), s));
  CK(cudaMemsetAsync(n->v, 0, NPARAM * sizeof(float), s));
  n->step = 0;
  int rc = refresh(n, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return XT_OK;
}

int xs_mlp_get_params(xs_mlp* n, float* params, int64_t count, void* stream) {
  g_err.clear();
  if (!n || !params || count != NPARAM) return fail(XT_ERR_INVALID, "need 202242 parameters");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(params, n->master, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return XT_OK;
}

int xs_mlp_forward(xs_mlp* n, const float* X, float* out, int64_t B, void* stream) {
  g_err.clear();
  if (!n || !X || !out || B < 0) return fail(XT_ERR_INVALID, "null argument or negative batch");
  if (B == 0) return XT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t CH = 65536;
  int rc = ensure_ws(n, std::min<int64_t>(B, CH));
  if (rc) return rc;
  for (int64_t o = 0; o < B; o += CH) {
    const int64_t b = std::min<int64_t>(CH, B - o);
    to_bf16_kernel<<<grid_1d(b * 16, 256), 256, 0, s>>>(X + o * 16, n->a[0], b * 16);
    CK(cudaGetLastError());
    bf16_t* acts[NL] = {n->a[0], n->a[1], n->a[2], n->a[1], n->a[2]};  // ping-pong
    rc = forward_layers(n, b, false, acts, out + 2 * o, s);
    if (rc) return rc;
  }
  return XT_OK;
}

int xs_mlp_loss_grad(xs_mlp* n, const float* X, const float* y, const float* t, const float* mask, int64_t B,
                     float lam, float* grad_out, float* loss_out, void* stream) {
  g_err.clear();
  if (!n || !X || !y || !t || !mask || B < 1) return fail(XT_ERR_INVALID, "null argument or empty batch");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = loss_grad(n, X, y, t, mask, B, lam, s);
  if (rc) return rc;
  if (grad_out) CK(cudaMemcpyAsync(grad_out, n->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (loss_out) CK(cudaMemcpyAsync(loss_out, n->scal, sizeof(float), cudaMemcpyDeviceToDevice, s));
  return XT_OK;
}

int xs_mlp_train_step(xs_mlp* n, const float* X, const float* y, const float* t, const float* mask, int64_t B,
                      float lr, float lam, float* loss_out, void* stream) {
  g_err.clear();
  if (!n || !X || !y || !t || !mask || B < 1) return fail(XT_ERR_INVALID, "null argument or empty batch");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = loss_grad(n, X, y, t, mask, B, lam, s);
  if (rc) return rc;
  n->step += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, (double)n->step));
  const float c2 = (float)(1.0 - std::pow(b2, (double)n->step));
  adam_kernel<<<grid_1d(NPARAM, 256), 256, 0, s>>>(n->master, n->grad, n->m, n->v, NPARAM, lr, (float)b1,
                                                   (float)b2, c1, c2, 1e-8f);
  CK(cudaGetLastError());
  rc = refresh(n, s);
  if (rc) return rc;
  if (loss_out) CK(cudaMemcpyAsync(loss_out, n->scal, sizeof(float), cudaMemcpyDeviceToDevice, s));
  return XT_OK;
}

const char* xs_last_error(void) { return g_err.c_str(); }

}  // extern "C"
