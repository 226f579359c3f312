// Glue of the surrogate-guided dynamic-aperture scan.
//
// The scan grid is ray-major: particle i = ray * n_r + k, radius index k
// increasing outward.  The dynamic aperture of a ray is read as the number of
// radii before the first particle that does not survive (scanning outward).
// The surrogate's survival logit locates where each ray's first loss is
// expected; a window of points around it is handed to the FP64 tracker by
// setting their state to 1 (tracked) and the others to XS_STATE_PREDICTED, so
// that xt_track's own compaction tracks only that band.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <string>

#include "xtgb.h"

namespace {
thread_local std::string g_err;

constexpr int DA_BLOCK = 256;  // one block per ray, threads over the radii

__device__ __forceinline__ int block_min(int v) {
  __shared__ int m;
  if (threadIdx.x == 0) m = INT_MAX;
  __syncthreads();
  v = __reduce_min_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) atomicMin(&m, v);
  __syncthreads();
  const int r = m;
  __syncthreads();
  return r;
}

// Per ray: r_lo = first k whose survival probability is below 1 - p_lo
// (logit < lmax), n_r if none: where the network first doubts survival, and
// so where the ray's first loss is expected.  First pass (widen == null): the
// window k in [r_lo - margin, r_lo + window] is tracked (state 1), every other
// point is predicted (XS_STATE_PREDICTED).  Later passes: survivors of the
// previous pass (state 1) become XS_STATE_SURVIVED so they are not tracked
// again, and predicted points are added next to the previous first loss dp:
// [dp - margin, dp - 1] on rays flagged XS_WIDEN_INWARD (the loss was tracked
// but its inner neighbour only predicted), [dp - margin, dp + margin] on rays
// flagged XS_WIDEN_VERIFY (the loss itself was only predicted).
__global__ void __launch_bounds__(DA_BLOCK) select_kernel(const float* __restrict__ out2, int32_t n_r, float lmax,
                                                          int32_t margin, int32_t window,
                                                          const int32_t* __restrict__ widen,
                                                          const int32_t* __restrict__ da_prev,
                                                          int32_t* __restrict__ state,
                                                          int32_t* __restrict__ r_lo_out) {
  const int ray = blockIdx.x;
  const int64_t base = (int64_t)ray * n_r;
  int first = n_r;
  for (int k = threadIdx.x; k < n_r; k += DA_BLOCK)
    if (out2[2 * (base + k)] < lmax) {
      first = k;
      break;
    }
  const int rl = block_min(first);
  if (threadIdx.x == 0) r_lo_out[ray] = rl;
  if (!widen) {
    const int lo = rl - margin, hi = rl + window;
    for (int k = threadIdx.x; k < n_r; k += DA_BLOCK)
      state[base + k] = (k >= lo && k <= hi) ? 1 : XS_STATE_PREDICTED;
    return;
  }
  const int w = widen[ray];
  const int dp = da_prev ? da_prev[ray] : rl;
  const int a = dp - margin;
  const int b = (w == XS_WIDEN_VERIFY) ? dp + margin : dp - 1;
  for (int k = threadIdx.x; k < n_r; k += DA_BLOCK) {
    int32_t s = state[base + k];
    if (s == 1) s = XS_STATE_SURVIVED;
    if (w != 0 && s == XS_STATE_PREDICTED && k >= a && k <= b) s = 1;
    state[base + k] = s;
  }
}

// Per ray: DA index = first k that is lost: a tracked point is lost if its
// state is <= 0, a predicted point if its logit < 0 (out2 may be null when
// every point was tracked).  widen[ray] = XS_WIDEN_VERIFY when that first
// loss is a predicted point, XS_WIDEN_INWARD when it is tracked but its inner
// neighbour was predicted (the boundary may lie further in), else 0.
__global__ void __launch_bounds__(DA_BLOCK) combine_kernel(const float* __restrict__ out2,
                                                           const int32_t* __restrict__ state, int32_t n_r,
                                                           int32_t* __restrict__ da, int32_t* __restrict__ widen) {
  const int ray = blockIdx.x;
  const int64_t base = (int64_t)ray * n_r;
  int first = n_r;
  for (int k = threadIdx.x; k < n_r; k += DA_BLOCK) {
    const int32_t s = state[base + k];
    const bool lost = (s == XS_STATE_PREDICTED) ? (out2 && out2[2 * (base + k)] < 0.f) : (s <= 0);
    if (lost) {
      first = k;
      break;
    }
  }
  first = block_min(first);
  if (threadIdx.x == 0) {
    int w = 0;
    if (first < n_r) {
      if (state[base + first] == XS_STATE_PREDICTED) w = XS_WIDEN_VERIFY;
      else if (first > 0 && state[base + first - 1] == XS_STATE_PREDICTED) w = XS_WIDEN_INWARD;
    }
    da[ray] = first;
    if (widen) widen[ray] = w;
  }
}
}  // namespace

extern "C" {

int xs_da_select(const float* out2, int32_t n_rays, int32_t n_r, float p_lo, int32_t margin, int32_t window,
                 const int32_t* widen, const int32_t* da_prev, int32_t* state, int32_t* r_lo, void* stream) {
  g_err.clear();
  if (!out2 || !state || !r_lo || n_rays < 0 || n_r < 0 || !(p_lo > 0.f && p_lo < 0.5f) || margin < 0 ||
      window < 0) {
    g_err = "xs_da_select: null pointer, p_lo outside (0, 0.5) or negative margin/window";
    return XT_ERR_INVALID;
  }
  if (n_rays == 0 || n_r == 0) return XT_OK;
  const float lmax = logf((1.0f - p_lo) / p_lo);
  select_kernel<<<n_rays, DA_BLOCK, 0, (cudaStream_t)stream>>>(out2, n_r, lmax, margin, window, widen, da_prev,
                                                              state, r_lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("xs_da_select: ") + cudaGetErrorString(e);
    return XT_ERR_CUDA;
  }
  return XT_OK;
}

int xs_da_combine(const float* out2, const int32_t* state, int32_t n_rays, int32_t n_r, int32_t* da,
                  int32_t* widen, void* stream) {
  g_err.clear();
  if (!state || !da || n_rays < 0 || n_r < 0) {
    g_err = "xs_da_combine: null pointer or negative size";
    return XT_ERR_INVALID;
  }
  if (n_rays == 0) return XT_OK;
  if (n_r == 0) {
    cudaError_t e = cudaMemsetAsync(da, 0, (size_t)n_rays * sizeof(int32_t), (cudaStream_t)stream);
    if (e == cudaSuccess && widen)
      e = cudaMemsetAsync(widen, 0, (size_t)n_rays * sizeof(int32_t), (cudaStream_t)stream);
    if (e != cudaSuccess) {
      g_err = std::string("xs_da_combine: ") + cudaGetErrorString(e);
      return XT_ERR_CUDA;
    }
    return XT_OK;
  }
  combine_kernel<<<n_rays, DA_BLOCK, 0, (cudaStream_t)stream>>>(out2, state, n_r, da, widen);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("xs_da_combine: ") + cudaGetErrorString(e);
    return XT_ERR_CUDA;
  }
  return XT_OK;
}

const char* xs_da_last_error(void) { return g_err.c_str(); }

}  // extern "C"
