// Dynamic-aperture surrogate network: MLP 16 -> 256 -> 256 -> 256 -> 256 -> 2
// (GELU, erf to 1.5e-7), BF16 weights and activations, FP32 accumulation in tensor
// memory on the tcgen05 tensor cores, FP32 master weights with Adam.
// Hand-written forward, backward and optimiser kernels.
//
// Rounding points (the oracle rounds at the same places): the network input,
// every weight matrix, every hidden activation and every back-propagated
// pre-activation gradient dZ are bfloat16; accumulations, biases, GELU and its
// derivative, the head (256 -> 2), the loss and Adam are FP32.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
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
// GELU(z) = z Phi(z) and GELU'(z) = Phi(z) + z phi(z), Phi the normal CDF,
// in FP32 from Hastings' rational approximation of erf (Abramowitz & Stegun
// 7.1.26): for x >= 0, erf(x) = 1 - t P(t) e^{-x^2} + eps with t = 1/(1 + p x),
// P a quartic, |eps| <= 1.5e-7.  With x = |z|/sqrt 2 the tail
// Phi(-|z|) = (1 - erf(x))/2 = t (P(t)/2) e^{-z^2/2}; then
// GELU(z) = max(z, 0) - |z| Phi(-|z|) for either sign of z, and
// Phi(z) = 1 - Phi(-|z|) for z >= 0, Phi(-|z|) otherwise.  The reciprocal and
// the exponential are the hardware approximations (rcp.approx, ex2.approx,
// relative errors near 2^-23); GELU is within 6e-7 |z| of its exact value and
// GELU' within 3e-7, far below the bfloat16 spacing of the activations.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// Phi(-|z|); *e receives exp(-z^2/2)
__device__ __forceinline__ float normal_tail(float z, float* e) {
  const float t = rcp_approx(fmaf(0.231641888f, fabsf(z), 1.0f));  // p / sqrt 2, p = 0.3275911
  float q = 0.5307027145f;                                          // a5 / 2
  q = fmaf(q, t, -0.7265760135f);                                   // a4 / 2
  q = fmaf(q, t, 0.7107068705f);                                    // a3 / 2
  q = fmaf(q, t, -0.142248368f);                                    // a2 / 2
  q = fmaf(q, t, 0.127414796f);                                     // a1 / 2
  *e = ex2_approx(z * (z * -0.72134752044448170f));                 // -log2(e) / 2
  return (q * t) * *e;
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  float e;
  const float tail = normal_tail(z, &e);
  const float phi = z >= 0.0f ? 1.0f - tail : tail;
  return fmaf(z * 0.39894228040143268f, e, phi);  // 1 / sqrt(2 pi)
}

// The same on two outputs at once: the packed FP32 pair instructions
// (fma/mul/add.rn.f32x2) do both lanes' arithmetic in one instruction with
// the rounding of the single-lane operations.
union F2 {
  float2 f;
  unsigned long long u;
};
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  F2 A, B, C, D;
  A.f = a; B.f = b; C.f = c;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D.u) : "l"(A.u), "l"(B.u), "l"(C.u));
  return D.f;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  F2 A, B, D;
  A.f = a; B.f = b;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(D.u) : "l"(A.u), "l"(B.u));
  return D.f;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  F2 A, B, D;
  A.f = a; B.f = b;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(D.u) : "l"(A.u), "l"(B.u));
  return D.f;
}
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 normal_tail2(float2 z, float2* e) {
  const float2 d = make_float2(fmaf(0.231641888f, fabsf(z.x), 1.0f), fmaf(0.231641888f, fabsf(z.y), 1.0f));
  const float2 t = make_float2(rcp_approx(d.x), rcp_approx(d.y));
  float2 q = fma2(splat2(0.5307027145f), t, splat2(-0.7265760135f));
  q = fma2(q, t, splat2(0.7107068705f));
  q = fma2(q, t, splat2(-0.142248368f));
  q = fma2(q, t, splat2(0.127414796f));
  const float2 a = mul2(mul2(z, z), splat2(-0.72134752044448170f));
  *e = make_float2(ex2_approx(a.x), ex2_approx(a.y));
  return mul2(mul2(q, t), *e);
}
__device__ __forceinline__ float2 gelu2(float2 z) {
  float2 e;
  const float2 tail = normal_tail2(z, &e);
  return make_float2(fmaf(-fabsf(z.x), tail.x, fmaxf(z.x, 0.0f)), fmaf(-fabsf(z.y), tail.y, fmaxf(z.y, 0.0f)));
}
__device__ __forceinline__ float2 gelu_grad2(float2 z) {
  float2 e;
  const float2 tail = normal_tail2(z, &e);
  const float2 phi = make_float2(z.x >= 0.0f ? 1.0f - tail.x : tail.x, z.y >= 0.0f ? 1.0f - tail.y : tail.y);
  return fma2(mul2(z, splat2(0.39894228040143268f)), e, phi);
}

// ---------------------------------------------------------------------------
// C[M x N] = A[M x K] * B[N x K]^T on the 5th-generation tensor cores
// (tcgen05): A, B bfloat16 with K contiguous, FP32 accumulator in tensor
// memory.  A tile is 128 rows x BN columns (BN = 64, or 16 for the narrow
// first-layer weight gradient) over a K slice of at most 256.  Operands
// arrive by TMA (cp.async.bulk.tensor) in 64-wide K blocks, one mbarrier per
// block, in the 128-byte-swizzled K-major layout the tensor cores read
// directly (rows of 128 bytes, 8-row groups 1024 bytes apart); K positions
// beyond the tensor are zero-filled by the copy engine, which also covers
// the 16-wide input layer and ragged tails.  One thread waits for each block
// and issues its K/16 tcgen05.mma; a commit to an mbarrier signals the
// accumulator.  CTAs are persistent over tiles (n fastest, so CTAs running
// together share rows of A); as soon as a tile's MMAs are done the next
// tile's operands are requested, and the copies overlap the epilogue: 8
// warps, two per group of 32 accumulator lanes (rows), read the accumulator
// with tcgen05.ld and apply the fused epilogue with 16-byte stores.  Two
// CTAs share an SM, so one CTA's MMAs also overlap the other's epilogue.
enum { EPI_GELU = 0, EPI_DGRAD = 1, EPI_F32ADD = 2 };
struct Epi {
  const float* bias;    // EPI_GELU
  float* z;             // EPI_GELU: pre-activation out (may be null); EPI_DGRAD: fp32 dZ out
  const float* zprev;   // EPI_DGRAD: pre-activation of this layer's output
  bf16_t* out_b;        // EPI_GELU: activation; EPI_DGRAD: bf16 dZ
  float* out_f;         // EPI_F32ADD
  float* colsum;        // EPI_DGRAD (may be null): column sums of the fp32 dZ added here (the bias gradient)
  bf16_t* out_bt;       // EPI_GELU, EPI_DGRAD (may be null): out_b transposed, element (row, col) at col * ldt + row
  int ld;               // leading dimension of every output / zprev (a multiple of 4)
  int ldt;              // leading dimension of out_bt (>= M)
  int* status;          // set to 1 if a tensor-core or copy wait gave up
};

constexpr int TC_M = 128, TC_BK = 64, TC_NST = 4, TC_KSLICE = TC_NST * TC_BK;
constexpr int64_t TC_WAIT_LIMIT = 2000000000LL;  // clock cycles, about one second

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzle layout: start address, 8-row groups 1024 bytes apart (the leading
// offset is not used by this layout), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > TC_WAIT_LIMIT) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

template <int CH>
__device__ __forceinline__ void tmem_load(uint32_t taddr, uint32_t* r);
template <>
__device__ __forceinline__ void tmem_load<32>(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
template <>
__device__ __forceinline__ void tmem_load<16>(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// A 16-column accumulator read issued without waiting, and the wait that
// completes it; the wait names the destination registers, so no use of them
// can be scheduled before it.
__device__ __forceinline__ void tmem_issue16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Epilogue of CH accumulator columns [col, col + CH) of one row; v receives
// the fp32 values written (EPI_DGRAD: dZ).
// SBIAS: the layer's bias is read from its copy in shared memory, sbias
template <int EPI, int CH, bool SBIAS = false>
__device__ __forceinline__ void epilogue(const Epi& e, int row, int col, const uint32_t* r, float* vout,
                                         const float* sbias = nullptr) {
  const int64_t o = (int64_t)row * e.ld + col;
  if (EPI == EPI_F32ADD) {
#pragma unroll
    for (int q = 0; q < CH / 4; q++)
      atomicAdd((float4*)(e.out_f + o + 4 * q),
                make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                            __uint_as_float(r[4 * q + 3])));
  } else {
    float v[CH];
#pragma unroll
    for (int q = 0; q < CH / 4; q++) {
      float4 a;
      if (EPI == EPI_GELU) a = SBIAS ? *((const float4*)(sbias + col) + q) : __ldg((const float4*)(e.bias + col) + q);
      else a = __ldg((const float4*)(e.zprev + o) + q);
      const float2 acc01 = make_float2(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]));
      const float2 acc23 = make_float2(__uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
      const float2 a01 = make_float2(a.x, a.y), a23 = make_float2(a.z, a.w);
      const float2 v01 = (EPI == EPI_GELU) ? add2(acc01, a01) : mul2(acc01, gelu_grad2(a01));
      const float2 v23 = (EPI == EPI_GELU) ? add2(acc23, a23) : mul2(acc23, gelu_grad2(a23));
      v[4 * q] = v01.x;
      v[4 * q + 1] = v01.y;
      v[4 * q + 2] = v23.x;
      v[4 * q + 3] = v23.y;
    }
    if (e.z) {
#pragma unroll
      for (int q = 0; q < CH / 4; q++)
        *(float4*)(e.z + o + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (EPI == EPI_DGRAD) {
#pragma unroll
      for (int i = 0; i < CH; i++) vout[i] = v[i];
    }
    uint32_t h[CH / 2];
#pragma unroll
    for (int i = 0; i < CH / 2; i++) {
      const float2 zi = make_float2(v[2 * i], v[2 * i + 1]);
      const float2 g = (EPI == EPI_GELU) ? gelu2(zi) : zi;
      h[i] = pack_bf16x2(g.x, g.y);
    }
#pragma unroll
    for (int q = 0; q < CH / 8; q++)
      *(uint4*)(e.out_b + o + 8 * q) = make_uint4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
    if (e.out_bt) {
      // the transposed copy the weight gradient reads (its K is the batch):
      // the warp's 32 lanes are 32 consecutive rows, so each column is one
      // contiguous 64-byte store
      bf16_t* t = e.out_bt + (int64_t)col * e.ldt + row;
#pragma unroll
      for (int i = 0; i < CH / 2; i++) {  // the packed pair's bits: column 2i low, 2i + 1 high
        t[(int64_t)(2 * i) * e.ldt] = (bf16_t)(h[i] & 0xFFFFu);
        t[(int64_t)(2 * i + 1) * e.ldt] = (bf16_t)(h[i] >> 16);
      }
    }
  }
}

// Sum over the warp's 32 lanes (rows) of each of 32 columns: a butterfly
// that halves the columns a lane keeps at every step (16 + 8 + 4 + 2 + 1
// shuffles), after which lane l holds column l; a fixed order, so the sums
// are reproducible.  Lane l then adds it to out[l].
__device__ __forceinline__ void warp_colsum32(float* v, int lane, float* out) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < off; j++) {
      const float send = upper ? v[j] : v[j + off];
      const float recv = __shfl_xor_sync(0xFFFFFFFFu, send, off);
      v[j] = (upper ? v[j + off] : v[j]) + recv;
    }
  }
  atomicAdd(out + lane, v[0]);
}

template <int EPI, int BN>
__global__ void __launch_bounds__(256, 2) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                      Epi e) {
  constexpr int A_BYTES = TC_M * TC_BK * 2, B_BYTES = BN * TC_BK * 2, STAGE = A_BYTES + B_BYTES;
  static_assert(STAGE % 1024 == 0, "stages must keep the 1024-byte alignment of the swizzle atoms");
  constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;
  constexpr int CH = BN < 32 ? BN : 32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TC_NST * STAGE);
  uint64_t* mma_bar = full + TC_NST;
  uint32_t* tslot = (uint32_t*)(mma_bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_mt = (M + TC_M - 1) / TC_M, n_nt = N / BN, n_ks = (K + TC_KSLICE - 1) / TC_KSLICE;
  const int n_tiles = n_mt * n_nt * n_ks;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_addr(tslot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int j = 0; j <= TC_NST; j++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(full + j)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  // instruction descriptor: D f32, A and B bf16, both K-major, N >> 3, M >> 4
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  auto coords = [&](int t, int& m0, int& n0, int& k0, int& k1) {
    const int nt = t % n_nt, mt = (t / n_nt) % n_mt, ks = t / (n_nt * n_mt);
    m0 = mt * TC_M;
    n0 = nt * BN;
    k0 = ks * TC_KSLICE;
    k1 = min(K, k0 + TC_KSLICE);
  };
  uint32_t pending = 0;  // K blocks with copies in flight (thread 0)
  auto request = [&](int t) {
    int m0, n0, k0, k1;
    coords(t, m0, n0, k0, k1);
    for (int j = 0; k0 + j * TC_BK < k1; j++) {
      const uint32_t bar = sm_addr(full + j);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(STAGE) : "memory");
      tma_load_2d(sm_addr(smem + j * STAGE), &tmA, k0 + j * TC_BK, m0, bar);
      tma_load_2d(sm_addr(smem + j * STAGE + A_BYTES), &tmB, k0 + j * TC_BK, n0, bar);
      pending |= 1u << j;
    }
  };
  uint32_t fphase = 0, mphase = 0;  // barrier parities (thread 0)
  int ok = 1, mma_open = 0;
  int t = blockIdx.x;
  if (tid == 0 && t < n_tiles) request(t);
  for (; t < n_tiles; t += gridDim.x) {
    int m0, n0, k0, k1;
    coords(t, m0, n0, k0, k1);
    if (tid == 0) {
      for (int j = 0; k0 + j * TC_BK < k1; j++) {
        if (!mbar_wait(sm_addr(full + j), (fphase >> j) & 1)) {
          ok = 0;
          break;
        }
        fphase ^= 1u << j;
        pending &= ~(1u << j);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int kc = min(TC_BK, k1 - (k0 + j * TC_BK));
        const uint64_t ad = smem_desc_sw128(sm_addr(smem + j * STAGE));
        const uint64_t bd = smem_desc_sw128(sm_addr(smem + j * STAGE + A_BYTES));
        for (int s = 0; s * 16 < kc; s++) {  // K = 16 per instruction: +32 bytes in the swizzled row
          const uint32_t accumulate = (j > 0 || s > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad + 2 * s), "l"(bd + 2 * s), "r"(idesc), "r"(accumulate)
              : "memory");
          mma_open = 1;
        }
      }
      if (ok) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         sm_addr(mma_bar))
                     : "memory");
        if (mbar_wait(sm_addr(mma_bar), mphase)) {
          mma_open = 0;
          mphase ^= 1;
        } else {
          ok = 0;
        }
      }
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the MMAs have read the operands: request the next tile's now, so the
    // copies run under this tile's epilogue
    if (tid == 0 && t + (int)gridDim.x < n_tiles) request(t + gridDim.x);
    // warps w and w + 4 share the 32 accumulator lanes (rows) of quadrant
    // w mod 4 and split the columns
    const int quad = warp & 3;
    const int row = m0 + quad * 32 + lane;
#pragma unroll 1
    for (int c0 = (warp >> 2) * CH; c0 < BN; c0 += 2 * CH) {
      uint32_t r[CH];
      tmem_load<CH>(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, r);
      float v[CH];
#pragma unroll
      for (int i = 0; i < CH; i++) v[i] = 0.0f;
      if (row < M) epilogue<EPI, CH>(e, row, n0 + c0, r, v);
      if constexpr (EPI == EPI_DGRAD && CH == 32) {
        if (e.colsum) warp_colsum32(v, lane, e.colsum + n0 + c0);  // rows past M add 0
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok && tid == 0) {
    if (e.status) atomicExch(e.status, 1);
    // let copies and MMAs still in flight finish (bounded) before the
    // shared and tensor memory are released
    for (int j = 0; j < TC_NST; j++)
      if (pending & (1u << j)) mbar_wait(sm_addr(full + j), (fphase >> j) & 1);
    if (mma_open) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       sm_addr(mma_bar))
                   : "memory");
      mbar_wait(sm_addr(mma_bar), mphase);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// Warp-specialised form of the same GEMM, for launches with many tiles per
// CTA: warp 0 issues the copies, warp 1 the MMAs, warps 2..9 run the
// epilogue.  mbarriers connect them: full[s] (copies landed) and empty[s]
// (the MMAs that read stage s are done) for the TC_NST operand stages, and
// accf[a] (MMAs of a tile done) and acce[a] (its accumulator read) for two
// accumulators in tensor memory.  The copies of later tiles, the MMAs of the
// next tile and the epilogue of this one therefore run at the same time.
// Every wait is clock-limited: a wait that gives up sets the CTA's error
// flag, every role leaves its loop, the copies and MMAs still in flight are
// waited for (again bounded), the tensor memory is freed and e.status is set.
constexpr int WS_THREADS = 320;
constexpr int WS_BIAS = 256;  // bias floats kept in shared memory

template <int EPI, int BN>
__global__ void __launch_bounds__(WS_THREADS) tc_gemm_ws_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, int M,
                                                                int N, int K, Epi e) {
  constexpr int A_BYTES = TC_M * TC_BK * 2, B_BYTES = BN * TC_BK * 2, STAGE = A_BYTES + B_BYTES;
  static_assert(STAGE % 1024 == 0, "stages must keep the 1024-byte alignment of the swizzle atoms");
  constexpr uint32_t ACC = BN < 32 ? 32 : BN;  // columns per accumulator
  constexpr uint32_t NCOLS = 2 * ACC;
  constexpr int CH = BN < 32 ? BN : 32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TC_NST * STAGE);
  uint64_t* empty = full + TC_NST;
  uint64_t* accf = empty + TC_NST;
  uint64_t* acce = accf + 2;
  uint64_t* drain = acce + 2;
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* err = (volatile int*)(tslot + 1);
  float* sbias = (float*)(smem + TC_NST * STAGE + 256);  // WS_BIAS floats
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_mt = (M + TC_M - 1) / TC_M, n_nt = N / BN, n_ks = (K + TC_KSLICE - 1) / TC_KSLICE;
  const int n_tiles = n_mt * n_nt * n_ks;
  // the bias is read once per CTA into shared memory (N <= WS_BIAS, checked
  // by the host)
  if (EPI == EPI_GELU) {
    for (int j = tid; j < N; j += WS_THREADS) sbias[j] = e.bias[j];
  }
  constexpr bool SB = EPI == EPI_GELU;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_addr(tslot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int j = 0; j < TC_NST; j++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(full + j)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(empty + j)) : "memory");
    }
    for (int a = 0; a < 2; a++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(accf + a)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(sm_addr(acce + a)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(drain)) : "memory");
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  auto coords = [&](int t, int& m0, int& n0, int& k0, int& k1) {
    const int nt = t % n_nt, mt = (t / n_nt) % n_mt, ks = t / (n_nt * n_mt);
    m0 = mt * TC_M;
    n0 = nt * BN;
    k0 = ks * TC_KSLICE;
    k1 = min(K, k0 + TC_KSLICE);
  };
  uint32_t armed = 0;  // warp 0, lane 0: stage fills issued
  int mma_open = 0;    // warp 1, lane 0: MMAs issued since the last commit that was waited for
  if (warp == 0) {
    if (lane == 0) {
      for (int t = blockIdx.x; t < n_tiles && !*err; t += gridDim.x) {
        int m0, n0, k0, k1;
        coords(t, m0, n0, k0, k1);
        for (int j = 0; k0 + j * TC_BK < k1; j++) {
          const int s = (int)(armed % TC_NST);
          const uint32_t ph = (armed / TC_NST) & 1u;
          if (!mbar_wait(sm_addr(empty + s), ph ^ 1u)) {
            *err = 1;
            break;
          }
          const uint32_t bar = sm_addr(full + s);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(STAGE) : "memory");
          tma_load_2d(sm_addr(smem + s * STAGE), &tmA, k0 + j * TC_BK, m0, bar);
          tma_load_2d(sm_addr(smem + s * STAGE + A_BYTES), &tmB, k0 + j * TC_BK, n0, bar);
          armed++;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0, i = 0;
      for (int t = blockIdx.x; t < n_tiles && !*err; t += gridDim.x, i++) {
        const uint32_t a = i & 1u, aph = (i >> 1) & 1u;
        if (!mbar_wait(sm_addr(acce + a), aph ^ 1u)) {
          *err = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        int m0, n0, k0, k1;
        coords(t, m0, n0, k0, k1);
        const uint32_t d = tmem + a * ACC;
        bool ok = true;
        for (int j = 0; k0 + j * TC_BK < k1; j++, it++) {
          const int s = (int)(it % TC_NST);
          if (!mbar_wait(sm_addr(full + s), (it / TC_NST) & 1u)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int kc = min(TC_BK, k1 - (k0 + j * TC_BK));
          const uint64_t ad = smem_desc_sw128(sm_addr(smem + s * STAGE));
          const uint64_t bd = smem_desc_sw128(sm_addr(smem + s * STAGE + A_BYTES));
          for (int q = 0; q * 16 < kc; q++) {
            const uint32_t accumulate = (j > 0 || q > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                "l"(ad + 2 * q), "l"(bd + 2 * q), "r"(idesc), "r"(accumulate)
                : "memory");
            mma_open = 1;
          }
          // the stage is free once these MMAs have read it
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           sm_addr(empty + s))
                       : "memory");
        }
        if (!ok) {
          *err = 1;
          break;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         sm_addr(accf + a))
                     : "memory");
      }
    }
  } else {
    const int quad = warp & 3;         // the accumulator lanes (rows) this warp may read
    const int half = (warp - 2) >> 2;  // 0 or 1: which columns
    uint32_t i = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, i++) {
      const uint32_t a = i & 1u, aph = (i >> 1) & 1u;
      int ok = mbar_wait(sm_addr(accf + a), aph) ? 1 : 0;
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (!ok) {
        *err = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int m0, n0, k0, k1;
      coords(t, m0, n0, k0, k1);
      const int row = m0 + quad * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + a * ACC;
      bool released = false;
#pragma unroll 1
      for (int c0 = half * CH; c0 < BN; c0 += 2 * CH) {
        uint32_t r[CH];
        float v[CH];
#pragma unroll
        for (int q = 0; q < CH; q++) v[q] = 0.0f;
        const bool last = c0 + 2 * CH >= BN;  // this warp's last read of the accumulator
        if constexpr (CH == 32) {
          // two 16-column reads: the second lands while the first is processed
          tmem_issue16(taddr + (uint32_t)c0, r);
          tmem_wait16(r);
          tmem_issue16(taddr + (uint32_t)c0 + 16u, r + 16);
          if (row < M) epilogue<EPI, 16, SB>(e, row, n0 + c0, r, v, sbias);
          __syncwarp();
          tmem_wait16(r + 16);
        } else {
          tmem_load<CH>(taddr + (uint32_t)c0, r);
        }
        if (last) {  // hand the accumulator back
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(acce + a)) : "memory");
          released = true;
        }
        if constexpr (CH == 32) {
          if (row < M) epilogue<EPI, 16, SB>(e, row, n0 + c0 + 16, r + 16, v + 16, sbias);
        } else {
          if (row < M) epilogue<EPI, CH, SB>(e, row, n0 + c0, r, v, sbias);
        }
        if constexpr (EPI == EPI_DGRAD && CH == 32) {
          if (e.colsum) warp_colsum32(v, lane, e.colsum + n0 + c0);  // rows past M add 0
        }
      }
      if (!released) {
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(acce + a)) : "memory");
      }
    }
  }
  __syncthreads();
  if (*err) {
    if (warp == 0 && lane == 0) {
      // the last fill of every stage has landed before the shared memory goes
      for (uint32_t s = 0; s < (uint32_t)TC_NST && s < armed; s++) {
        const uint32_t last = s + ((armed - 1 - s) / TC_NST) * TC_NST;
        mbar_wait(sm_addr(full + s), (last / TC_NST) & 1u);
      }
    }
    if (warp == 1 && lane == 0 && mma_open) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       sm_addr(drain))
                   : "memory");
      mbar_wait(sm_addr(drain), 0);
    }
    if (tid == 0 && e.status) atomicExch(e.status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// rows x cols bfloat16, row stride ld elements; boxes of 64 columns x box_rows
// rows in the 128-byte swizzle, zero fill outside the tensor.
int make_tensor_map(CUtensorMap* m, const bf16_t* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(XT_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  if (((uintptr_t)ptr & 15) || (ld * 2) % 16 || rows < 1 || cols < 1)
    return fail(XT_ERR_INVALID, "tensor map: base must be 16-byte aligned and the row stride a multiple of 16 bytes");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)ptr, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(XT_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return XT_OK;
}

int sm_count_of_current_device() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
  return cache[dev];
}

template <int EPI, int BN>
int tc_launch(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, const Epi& e, cudaStream_t s) {
  constexpr size_t smem = (size_t)TC_NST * (TC_M * TC_BK * 2 + BN * TC_BK * 2) + 1024 + 256;
  static int occ = 0;
  if (!occ) {
    CK(cudaFuncSetAttribute(tc_gemm_kernel<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CK(cudaFuncSetAttribute(tc_gemm_kernel<EPI, BN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                            (int)cudaSharedmemCarveoutMaxShared));
    // CTAs per SM from the shared memory (with the per-block reservation) and
    // the 512 tensor-memory columns; the CTAs of the persistent grid never wait
    // on one another, so launching more than fit at once is only slower
    int dev = 0, per_sm = 0, reserved = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    const int by_smem = per_sm / (int)(smem + (size_t)reserved);
    occ = std::max(1, std::min(by_smem, 512 / (BN < 32 ? 32 : BN)));
  }
  const int64_t tiles = (int64_t)((M + TC_M - 1) / TC_M) * (N / BN) * ((K + TC_KSLICE - 1) / TC_KSLICE);
  const int sms = sm_count_of_current_device();
  if (sms <= 0) return fail(XT_ERR_CUDA, "device attribute");
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)occ * sms);
  tc_gemm_kernel<EPI, BN><<<grid, 256, smem, s>>>(ta, tb, M, N, K, e);
  CK(cudaGetLastError());
  return XT_OK;
}

// The warp-specialised kernel for the same tiles, when there are more tiles
// than resident CTAs (each CTA then pipelines several).
template <int EPI, int BN>
int tc_launch_ws(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, const Epi& e, cudaStream_t s) {
  constexpr size_t smem =
      (size_t)TC_NST * (TC_M * TC_BK * 2 + BN * TC_BK * 2) + 1024 + 256 + WS_BIAS * sizeof(float);
  static int occ = 0;
  if (!occ) {
    CK(cudaFuncSetAttribute(tc_gemm_ws_kernel<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CK(cudaFuncSetAttribute(tc_gemm_ws_kernel<EPI, BN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                            (int)cudaSharedmemCarveoutMaxShared));
    int dev = 0, per_sm = 0, reserved = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    const int by_smem = per_sm / (int)(smem + (size_t)reserved);
    occ = std::max(1, std::min(by_smem, 512 / (2 * (BN < 32 ? 32 : BN))));
  }
  const int64_t tiles = (int64_t)((M + TC_M - 1) / TC_M) * (N / BN) * ((K + TC_KSLICE - 1) / TC_KSLICE);
  const int sms = sm_count_of_current_device();
  if (sms <= 0) return fail(XT_ERR_CUDA, "device attribute");
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)occ * sms);
  tc_gemm_ws_kernel<EPI, BN><<<grid, WS_THREADS, smem, s>>>(ta, tb, M, N, K, e);
  CK(cudaGetLastError());
  return XT_OK;
}

// C = A B^T: A (M x K, row stride lda), B (N x K, row stride ldb), N = 256 or
// 16 (16 only for the split-K weight gradient).  K slices of 256 run in
// separate CTAs; EPI_F32ADD adds their partial sums into a zeroed output,
// the other epilogues need K <= 256.
template <int EPI>
int gemm(const bf16_t* A, int lda, const bf16_t* B, int ldb, int M, int N, int K, const Epi& e, cudaStream_t s) {
  if (M <= 0) return XT_OK;
  if (K < 1 || (K > TC_KSLICE && EPI != EPI_F32ADD) || e.ld % 4)
    return fail(XT_ERR_INVALID, "gemm: K must be in 1..256 for this epilogue and ld a multiple of 4");
  alignas(64) CUtensorMap ta, tb;
  int rc = make_tensor_map(&ta, A, M, K, lda, TC_M);
  if (rc) return rc;
  if (N == 256) {
    rc = make_tensor_map(&tb, B, N, K, ldb, 64);
    if (rc) return rc;
    // more tiles than two per SM: the warp-specialised pipeline
    const int64_t tiles = (int64_t)((M + TC_M - 1) / TC_M) * (N / 64) * ((K + TC_KSLICE - 1) / TC_KSLICE);
    if (tiles > 2 * (int64_t)sm_count_of_current_device() && (EPI != EPI_GELU || N <= WS_BIAS))
      return tc_launch_ws<EPI, 64>(ta, tb, M, N, K, e, s);
    return tc_launch<EPI, 64>(ta, tb, M, N, K, e, s);
  }
  if constexpr (EPI == EPI_F32ADD) {
    if (N == 16) {
      rc = make_tensor_map(&tb, B, N, K, ldb, 16);
      if (rc) return rc;
      return tc_launch<EPI, 16>(ta, tb, M, N, K, e, s);
    }
  }
  return fail(XT_ERR_INVALID, "gemm: unsupported N");
}

// ---------------------------------------------------------------------------
__global__ void to_bf16_kernel(const float* __restrict__ x, bf16_t* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = f2bf(x[i]);
}

// The 16-wide input batch in bf16, row-major (y) and transposed (yt, row c
// of length ldt holds column c), for training.
__global__ void to_bf16_t_kernel(const float* __restrict__ x, bf16_t* __restrict__ y, bf16_t* __restrict__ yt,
                                 int64_t B, int64_t ldt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * 16;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bf16_t h = f2bf(x[i]);
    y[i] = h;
    yt[(i & 15) * ldt + (i >> 4)] = h;
  }
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

// Head backward: dW5, db5 (atomics over batch slices), dZ4, its transpose
// (dzT, leading dimension ldt, for the weight gradient) and its column sums
// (the top hidden layer's bias gradient).  A block takes HB_TILE samples at
// a time and stages their bf16 dZ in shared memory, so that each transposed
// row goes out as one contiguous 16-byte piece.
constexpr int HB_TILE = 8;
__global__ void head_backward_kernel(const float* __restrict__ dout, const bf16_t* __restrict__ a4,
                                     const bf16_t* __restrict__ w5, const float* __restrict__ z4, int64_t B,
                                     float* __restrict__ gw5, float* __restrict__ gb5, float* __restrict__ dzf,
                                     bf16_t* __restrict__ dzb, float* __restrict__ gb4, bf16_t* __restrict__ dzT,
                                     int64_t ldt) {
  __shared__ __align__(16) bf16_t tile[256][HB_TILE];
  const int k = threadIdx.x;  // 256 threads: one hidden unit each
  const float w0 = bf2f(w5[k]), w1 = bf2f(w5[256 + k]);
  float s0 = 0.f, s1 = 0.f, d0 = 0.f, d1 = 0.f, sb = 0.f;
  for (int64_t b0 = (int64_t)blockIdx.x * HB_TILE; b0 < B; b0 += (int64_t)gridDim.x * HB_TILE) {
#pragma unroll
    for (int j = 0; j < HB_TILE; j++) {
      const int64_t b = b0 + j;
      bf16_t hb = f2bf(0.0f);
      if (b < B) {
        const float g0 = dout[2 * b], g1 = dout[2 * b + 1];
        const float a = bf2f(a4[b * 256 + k]);
        s0 = fmaf(g0, a, s0);
        s1 = fmaf(g1, a, s1);
        if (k == 0) { d0 += g0; d1 += g1; }
        const float dz = (g0 * w0 + g1 * w1) * gelu_grad_f(z4[b * 256 + k]);
        dzf[b * 256 + k] = dz;
        hb = f2bf(dz);
        dzb[b * 256 + k] = hb;
        sb += dz;
      }
      tile[k][j] = hb;
    }
    __syncthreads();
    // row r of dzT gets tile[r][0 .. HB_TILE): thread k writes row k (ldt and
    // b0 are multiples of 8, so the piece is 16-byte aligned; a piece past
    // ldt is never written because ldt is a multiple of 16 >= B)
    if (b0 + HB_TILE <= ldt) *(uint4*)(dzT + (int64_t)k * ldt + b0) = *(const uint4*)&tile[k][0];
    __syncthreads();
  }
  atomicAdd(&gb4[k], sb);  // the top hidden layer's bias gradient
  atomicAdd(&gw5[k], s0);
  atomicAdd(&gw5[256 + k], s1);
  if (k == 0) {
    atomicAdd(&gb5[0], d0);
    atomicAdd(&gb5[1], d1);
  }
}

// Adam on the fp32 master parameters, and in the same pass the bfloat16
// copies of every weight the next step's GEMMs read: W (out x in) and its
// transpose (in x out), which the separate refresh pass wrote before.
__constant__ int64_t c_off_w[NL] = {OFF_W[0], OFF_W[1], OFF_W[2], OFF_W[3], OFF_W[4]};
__constant__ int c_width[NL + 1] = {WIDTH[0], WIDTH[1], WIDTH[2], WIDTH[3], WIDTH[4], WIDTH[5]};
__global__ void adam_refresh_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                    float* __restrict__ v, int64_t n, float lr, float b1, float b2, float c1,
                                    float c2, float eps, bf16_t* __restrict__ wb, bf16_t* __restrict__ wtb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
#pragma unroll
    for (int l = 0; l < NL; l++) {
      const int out = c_width[l + 1], in = c_width[l];
      const int64_t j = i - c_off_w[l];
      if (j >= 0 && j < (int64_t)out * in) {
        const bf16_t h = f2bf(wi);
        wb[i] = h;
        wtb[c_off_w[l] + (j % in) * out + j / in] = h;
      }
    }
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
  bf16_t* dzT = nullptr;        // dZ transposed (256 x Bp), for the weight gradient
  bf16_t* aT[NL - 1] = {nullptr};  // a0 .. a3 transposed (in x Bp), for the weight gradient
};

static void free_ws(xs_mlp* n) {
  for (int i = 0; i < NL; i++) { cudaFree(n->a[i]); n->a[i] = nullptr; }
  for (int i = 0; i < NL - 1; i++) { cudaFree(n->z[i]); n->z[i] = nullptr; }
  for (int i = 0; i < 2; i++) { cudaFree(n->dzf[i]); cudaFree(n->dzb[i]); n->dzf[i] = nullptr; n->dzb[i] = nullptr; }
  cudaFree(n->out); cudaFree(n->dout); cudaFree(n->dzT);
  for (int i = 0; i < NL - 1; i++) { cudaFree(n->aT[i]); n->aT[i] = nullptr; }
  n->out = n->dout = nullptr;
  n->dzT = nullptr;
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
  for (int i = 0; i < NL - 1; i++) CK(cudaMalloc(&n->aT[i], (size_t)Bp * WIDTH[i] * sizeof(bf16_t)));
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
    // training: the transposed activations a1 .. a3 for the weight gradients
    e.out_bt = (keep_z && l + 1 < NL - 1) ? n->aT[l + 1] : nullptr;
    e.ldt = (int)pad16(B);
    e.ld = 256;
    e.status = (int*)(n->scal + 3);
    const int rc = gemm<EPI_GELU>(acts[l], WIDTH[l], n->wb + OFF_W[l], WIDTH[l], (int)B, 256, WIDTH[l], e, s);
    if (rc) return rc;
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
  const int64_t Bp = pad16(B);
  to_bf16_t_kernel<<<grid_1d(B * 16, 256), 256, 0, s>>>(X, n->a[0], n->aT[0], B, Bp);
  CK(cudaGetLastError());
  rc = forward_layers(n, B, true, n->a, n->out, s);
  if (rc) return rc;
  CK(cudaMemsetAsync(n->scal, 0, 2 * sizeof(float), s));  // loss, mask count (scal[3]: status)
  mask_count_kernel<<<grid_1d(B, 256), 256, 0, s>>>(mask, B, n->scal + 1);
  loss_kernel<<<grid_1d(B, 256), 256, 0, s>>>(n->out, y, t, mask, B, lam, n->dout, n->scal);
  CK(cudaMemsetAsync(n->grad, 0, NPARAM * sizeof(float), s));
  const int hb = (int)std::min<int64_t>((B + HB_TILE - 1) / HB_TILE, 1024);
  head_backward_kernel<<<hb, 256, 0, s>>>(n->dout, n->a[NL - 1], n->wb + OFF_W[NL - 1], n->z[NL - 2], B,
                                          n->grad + OFF_W[NL - 1], n->grad + OFF_B[NL - 1], n->dzf[0], n->dzb[0],
                                          n->grad + OFF_B[NL - 2], n->dzT, Bp);
  CK(cudaGetLastError());
  int cur = 0;
  for (int l = NL - 2; l >= 0; l--) {
    const int in = WIDTH[l];
    // wgrad: dW_l = dZ^T a_l (M = 256 outputs, N = in, K = the batch), from
    // the transposed copies that the producers of dZ and a_l wrote; the
    // tensor maps end K at B, so the copy engine zero-fills the padding
    Epi e;
    std::memset(&e, 0, sizeof(e));
    e.out_f = n->grad + OFF_W[l];
    e.ld = in;
    e.status = (int*)(n->scal + 3);
    // K (the batch) is split in slices of 256 whose partial sums add up in the gradient
    rc = gemm<EPI_F32ADD>(n->dzT, (int)Bp, n->aT[l], (int)Bp, 256, in, (int)B, e, s);
    if (rc) return rc;
    // the bias gradient of layer l (column sums of its fp32 dZ) was added by
    // the kernel that produced dZ: head_backward_kernel or the dgrad epilogue
    if (l > 0) {
      // dgrad: dA_{l-1} = dZ_l W_l, then times GELU'(z_{l-1})
      Epi d;
      std::memset(&d, 0, sizeof(d));
      d.zprev = n->z[l - 1];
      d.z = n->dzf[1 - cur];
      d.out_b = n->dzb[1 - cur];
      d.colsum = n->grad + OFF_B[l - 1];
      d.out_bt = n->dzT;  // read by the next weight gradient, after this one's
      d.ldt = (int)Bp;
      d.ld = 256;
      d.status = (int*)(n->scal + 3);
      rc = gemm<EPI_DGRAD>(n->dzb[cur], 256, n->wtb + OFF_W[l], 256, (int)B, 256, 256, d, s);
      if (rc) return rc;
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
  if (cudaMemset(n->scal, 0, 4 * sizeof(float)) != cudaSuccess) return bail(fail(XT_ERR_CUDA, "cudaMemset"));
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
  int32_t st = 0;
  CK(cudaMemcpyAsync(&st, n->scal + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st) return fail(XT_ERR_TIMEOUT, "a tensor-core wait gave up in an earlier network kernel");
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
  adam_refresh_kernel<<<grid_1d(NPARAM, 256), 256, 0, s>>>(n->master, n->grad, n->m, n->v, NPARAM, lr, (float)b1,
                                                           (float)b2, c1, c2, 1e-8f, n->wb, n->wtb);
  CK(cudaGetLastError());
  if (loss_out) CK(cudaMemcpyAsync(loss_out, n->scal, sizeof(float), cudaMemcpyDeviceToDevice, s));
  return XT_OK;
}

const char* xs_last_error(void) { return g_err.c_str(); }

}  // extern "C"
