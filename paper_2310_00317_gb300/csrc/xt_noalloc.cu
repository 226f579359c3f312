// xt_track_noalloc: tracking without any device allocation.
//
// xt_track keeps a per-tracker workspace (alive-index list, block counts,
// work counter, status) that it grows with cudaMalloc the first time it sees a
// larger particle count.  Some callers cannot allocate device memory while
// they track: host applications whose device memory is owned by their own
// allocator or budget and that forbid cudaMalloc after start-up, and real-time
// loops that cannot afford allocation latency or the device-wide
// synchronisation cudaMalloc and cudaFree can imply.  For them this entry point uses
// a fixed scratch array in static device memory instead: every GPU that loads
// the library holds it (about 4 MiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "xt_internal.h"

namespace {

// Scratch layout, in int32 words: [alive index list: MAX] [block counts:
// MAX/1024 + 1] [status, alive count, work counter, ...: 64].
constexpr int64_t NOALLOC_MAX = XT_NOALLOC_MAX_PARTICLES;
constexpr int64_t COUNTS_OFF = NOALLOC_MAX;
constexpr int64_t SCAL_OFF = COUNTS_OFF + NOALLOC_MAX / 1024 + 64;
constexpr int64_t SCRATCH_WORDS = SCAL_OFF + 64;

static __device__ __align__(256) int32_t g_noalloc_scratch[SCRATCH_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
int32_t* g_ptr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not a device address).
int scratch_for_current_device(int32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    xt::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return XT_ERR_CUDA;
  }
  if (dev < 0 || dev >= MAX_DEVICES) {
    xt::set_error("xt_track_noalloc supports device ordinals below 64");
    return XT_ERR_INVALID;
  }
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      xt::set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return XT_ERR_CUDA;
    }
    g_ptr[dev] = (int32_t*)p;
  }
  *out = g_ptr[dev];
  return XT_OK;
}

}  // namespace

extern "C" int xt_track_noalloc(xt_tracker* tr, const xt_particles* p, int64_t start_turn, int64_t n_turns,
                                void* stream) {
  xt::set_error("");
  if (!tr || !p) {
    xt::set_error("tracker or particles is null");
    return XT_ERR_INVALID;
  }
  if (p->n < 0 || p->n > NOALLOC_MAX) {
    xt::set_error("xt_track_noalloc handles at most " + std::to_string(NOALLOC_MAX) +
                  " particles per call (got " + std::to_string(p->n) + "); use xt_track for more");
    return XT_ERR_INVALID;
  }
  if (start_turn < 0 || n_turns < 0 || start_turn + n_turns > 0x7fffffff) {
    xt::set_error("turn range outside 0..2^31-1");
    return XT_ERR_INVALID;
  }
  if (p->n > 0) {
    const void* ptrs[] = {p->x, p->px, p->y, p->py, p->zeta, p->delta, p->ptau, p->rpp, p->rvv,
                          p->state, p->at_turn, p->at_element, p->particle_id};
    for (const void* q : ptrs) {
      if (!q) {
        xt::set_error("particle arrays are null");
        return XT_ERR_INVALID;
      }
    }
  }
  if (p->n == 0 || n_turns == 0) return XT_OK;
  int32_t* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  xt::TrackArgs a;
  int block = 0, grid = 0, seg = 1, rad = 0;
  size_t smem = 0;
  rc = xt::noalloc_prepare(tr, p, n_turns, &a, &block, &grid, &smem, &seg, &rad);
  if (rc) return rc;
  int32_t* idx = scratch;
  int32_t* counts = scratch + COUNTS_OFF;
  int32_t* scal = scratch + SCAL_OFF;  // [0] status [1] alive count [2] work counter
  a.idx = idx;
  a.status = scal;
  a.n_alive = scal + 1;
  a.tile_counter = scal + 2;
  // The array keeps the previous call's contents: the status word must start at 0.
  cudaError_t e = cudaMemsetAsync(scal, 0, sizeof(int32_t), (cudaStream_t)stream);
  if (e != cudaSuccess) {
    xt::set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    return XT_ERR_CUDA;
  }
  for (int64_t done = 0; done < n_turns; done += seg) {
    const int nt = (int)((n_turns - done) < seg ? (n_turns - done) : seg);
    int le = xt::launch_compact(p->state, p->n, counts, idx, scal + 1, scal + 2, stream);
    if (le) {
      xt::set_error(std::string("compaction launch: ") + cudaGetErrorString((cudaError_t)le));
      return XT_ERR_CUDA;
    }
    a.turn0 = (int32_t)(start_turn + done);
    a.n_turns = nt;
    le = xt::launch_track(a, rad, block, grid, smem, stream);
    if (le) {
      xt::set_error(std::string("tracking launch: ") + cudaGetErrorString((cudaError_t)le));
      return XT_ERR_CUDA;
    }
  }
  return XT_OK;
}

// Status word of the scratch array on the current device: the outcome of the
// last xt_track_noalloc call there (XT_OK, XT_ERR_TIMEOUT or
// XT_ERR_CANCELLED).  Synchronises the stream, reads the word and clears it.
extern "C" int xt_noalloc_status(void* stream) {
  xt::set_error("");
  int32_t* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  int32_t st = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&st, scratch + SCAL_OFF, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch + SCAL_OFF, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    xt::set_error(std::string("xt_noalloc_status: ") + cudaGetErrorString(e));
    return XT_ERR_CUDA;
  }
  return st;
}
