// C ABI of the tracker: lattice compilation, device buffers, segmented
// launches with compaction, the host-buffer path, the autotuner and the
// batched-seed launch captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "xt_internal.h"

using namespace xt;

// Frees the batched plans that name a tracker (defined with the plans below).
void evict_plans_of(const xt_tracker* t);

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return XT_ERR_CUDA;
}
#define CK(call)                                              \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return cuda_fail(_e, #call);       \
  } while (0)

const int DEFAULT_BLOCK = 128;
const int DEFAULT_CHUNK = 4096;

int check_options(const xt_options& o) {
  if (o.radiation < 0 || o.radiation > 2) return fail(XT_ERR_INVALID, "radiation must be 0, 1 or 2");
  if (o.block != 0 && (o.block < 32 || o.block > 256 || o.block % 32))
    return fail(XT_ERR_INVALID, "block must be 0 or a multiple of 32 in 32..256");
  if (o.chunk_bytes != 0 && (o.chunk_bytes < 1024 || o.chunk_bytes > 49152 || o.chunk_bytes % 16))
    return fail(XT_ERR_INVALID, "chunk_bytes must be 0 or a multiple of 16 in 1024..49152");
  if (o.segment_turns < 0) return fail(XT_ERR_INVALID, "segment_turns must be >= 0");
  if (o.max_cycles < 0) return fail(XT_ERR_INVALID, "max_cycles must be >= 0");
  return XT_OK;
}

bool particles_ok(const xt_particles* p) {
  if (!p || p->n < 0 || p->n > 0x7fffffff) return false;
  if (p->n == 0) return true;
  const void* ptrs[] = {p->x, p->px, p->y, p->py, p->zeta, p->delta, p->ptau, p->rpp, p->rvv,
                        p->state, p->at_turn, p->at_element, p->particle_id};
  for (const void* q : ptrs)
    if (!q) return false;
  return true;
}

template <class T>
int dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    g_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? XT_ERR_NOMEM : XT_ERR_CUDA;
  }
  return XT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
struct xt_tracker {
  Lattice lat;
  Refc rc;
  RefDev ref;
  SinTab sn;
  xt_options opt;
  int device = 0;
  int sm_count = 1;
  int smem_max = 0;
  std::vector<xt_element> table;  // kept for flop accounting
  uint8_t* d_lat = nullptr;
  Chunk* d_chunks = nullptr;
  int n_chunks = 0;
  int chunk_built = 0;  // chunk size the table was built for
  double* d_spec_xi = nullptr;
  double* d_spec_F = nullptr;
  int32_t* d_spec_guide = nullptr;
  int spec_k = 0;
  int32_t* d_scal = nullptr;  // [0] status [1] n_alive [2] tile_counter [3] turn base
  int32_t* h_cancel = nullptr;
  int32_t* d_cancel = nullptr;
  // workspace
  int32_t* d_idx = nullptr;
  int32_t* d_counts = nullptr;
  int64_t ws_n = -1;
  // device copies for the host-buffer path
  void* d_stage = nullptr;
  int64_t stage_n = -1;
  // optional event timing of the tracking kernel launches
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t ev_used = 0;
  // loss-location refinement tables (one device buffer), built on first use
  int refine_angles = 0;
  uint8_t* d_refine = nullptr;
  RefineArgs refine_tab;  // table pointers into d_refine
  // per-row record offsets for the monitor, uploaded on first use
  int32_t* d_rowoff = nullptr;
};

// Kernel instantiation for a tracker: radiation mode + 3 if its table has
// thick rows (the thin-only instantiation leaves their code out of the loop).
static int kind_of(const xt_tracker* t) { return t->opt.radiation + (t->lat.thick ? 3 : 0); }

static int prof_pair(xt_tracker* t, cudaEvent_t* a, cudaEvent_t* b) {
  if (t->ev_used == t->ev.size()) {
    cudaEvent_t x, y;
    CK(cudaEventCreate(&x));
    CK(cudaEventCreate(&y));
    t->ev.push_back({x, y});
  }
  *a = t->ev[t->ev_used].first;
  *b = t->ev[t->ev_used].second;
  t->ev_used++;
  return XT_OK;
}

static int build_device_chunks(xt_tracker* t, int chunk_bytes) {
  if (t->chunk_built == chunk_bytes && t->d_chunks) return XT_OK;
  std::vector<Chunk> ch;
  build_chunks(t->lat, (uint32_t)chunk_bytes, &ch);
  for (const Chunk& c : ch)
    if (c.bytes > (uint32_t)chunk_bytes)
      return fail(XT_ERR_INVALID, "chunk_bytes smaller than one lattice record");
  if (t->d_chunks) cudaFree(t->d_chunks);
  t->d_chunks = nullptr;
  int rc = dev_alloc(&t->d_chunks, ch.size());
  if (rc) return rc;
  if (!ch.empty()) CK(cudaMemcpy(t->d_chunks, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
  t->n_chunks = (int)ch.size();
  t->chunk_built = chunk_bytes;
  return XT_OK;
}

static int eff_block(const xt_tracker* t) { return t->opt.block ? t->opt.block : DEFAULT_BLOCK; }
static int eff_chunk(const xt_tracker* t) { return t->opt.chunk_bytes ? t->opt.chunk_bytes : DEFAULT_CHUNK; }
static int eff_segment(const xt_tracker* t, int64_t n, int64_t n_turns) {
  if (t->opt.segment_turns > 0) return (int)std::min<int64_t>(t->opt.segment_turns, std::max<int64_t>(n_turns, 1));
  // aim for >= ~1e8 particle-element passes per launch so launch overhead stays small
  const double work = (double)std::max<int64_t>(n, 1) * (double)std::max<int64_t>(t->lat.n_el, 1);
  int64_t s = (int64_t)(1e8 / work) + 1;
  return (int)std::max<int64_t>(1, std::min<int64_t>(s, std::max<int64_t>(n_turns, 1)));
}

static int ensure_workspace(xt_tracker* t, int64_t n) {
  if (n <= t->ws_n) return XT_OK;
  if (t->d_idx) cudaFree(t->d_idx);
  if (t->d_counts) cudaFree(t->d_counts);
  t->d_idx = nullptr;
  t->d_counts = nullptr;
  t->ws_n = -1;
  int rc = dev_alloc(&t->d_idx, (size_t)n);
  if (rc) return rc;
  rc = dev_alloc(&t->d_counts, (size_t)((n + 1023) / 1024 + 1));
  if (rc) return rc;
  t->ws_n = n;
  return XT_OK;
}

static void fill_args(const xt_tracker* t, const xt_particles* p, TrackArgs* a) {
  std::memset(a, 0, sizeof(*a));
  a->lat = t->d_lat;
  a->chunks = t->d_chunks;
  a->n_chunks = t->n_chunks;
  a->n_el = (int32_t)t->lat.n_el;
  a->chunk_bytes = t->chunk_built;
  a->x = p->x; a->px = p->px; a->y = p->y; a->py = p->py; a->zeta = p->zeta;
  a->delta = p->delta; a->ptau = p->ptau; a->rpp = p->rpp; a->rvv = p->rvv;
  a->state = p->state; a->at_turn = p->at_turn; a->at_element = p->at_element;
  a->pid = p->particle_id;
  a->idx = t->d_idx;
  a->n_alive = t->d_scal + 1;
  a->tile_counter = t->d_scal + 2;
  a->status = t->d_scal;
  a->cancel = t->d_cancel;
  a->max_cycles = t->opt.max_cycles;
  a->seed = t->opt.seed;
  a->spec_xi = t->d_spec_xi;
  a->spec_F = t->d_spec_F;
  a->spec_guide = t->d_spec_guide;
  a->spec_k = t->spec_k;
  a->ref = t->ref;
  a->sn = t->sn;
}

static int grid_for(xt_tracker* t, int block, size_t smem, int* grid) {
  if (smem > (size_t)t->smem_max)
    return fail(XT_ERR_INVALID, "block x 2 x chunk_bytes exceeds the shared memory of one block (" +
                                    std::to_string(smem) + " > " + std::to_string(t->smem_max) + ")");
  int bps = 0;
  int e = track_occupancy(kind_of(t), block, smem, &bps);
  if (e) return cuda_fail((cudaError_t)e, "occupancy");
  if (bps < 1) return fail(XT_ERR_INVALID, "launch configuration does not fit on an SM");
  *grid = bps * t->sm_count;
  return XT_OK;
}

static int track_device(xt_tracker* t, const xt_particles* p, int64_t start_turn, int64_t n_turns,
                        void* stream) {
  if (p->n == 0 || n_turns == 0) return XT_OK;
  int rc = ensure_workspace(t, p->n);
  if (rc) return rc;
  const int block = eff_block(t);
  rc = build_device_chunks(t, eff_chunk(t));
  if (rc) return rc;
  const size_t smem = track_smem_bytes(block, t->chunk_built, kind_of(t));
  int grid = 0;
  rc = grid_for(t, block, smem, &grid);
  if (rc) return rc;
  const int seg = eff_segment(t, p->n, n_turns);
  TrackArgs a;
  fill_args(t, p, &a);
  for (int64_t done = 0; done < n_turns; done += seg) {
    const int nt = (int)std::min<int64_t>(seg, n_turns - done);
    int e = launch_compact(p->state, p->n, t->d_counts, t->d_idx, t->d_scal + 1, t->d_scal + 2, stream);
    if (e) return cuda_fail((cudaError_t)e, "compaction launch");
    a.turn0 = (int32_t)(start_turn + done);
    a.n_turns = nt;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (t->prof) {
      rc = prof_pair(t, &ea, &eb);
      if (rc) return rc;
      CK(cudaEventRecord(ea, (cudaStream_t)stream));
    }
    e = launch_track(a, kind_of(t), block, grid, smem, stream);
    if (e) return cuda_fail((cudaError_t)e, "tracking launch");
    if (t->prof) CK(cudaEventRecord(eb, (cudaStream_t)stream));
  }
  return XT_OK;
}

extern "C" {

void xt_options_default(xt_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->radiation = XT_RAD_OFF;
}

const char* xt_last_error(void) { return g_err.c_str(); }
const char* xt_version(void) { return "xtgb 0.1 (sm_103a, FP64)"; }

int xt_tracker_create(const xt_element* table, int64_t n, const xt_reference* ref, const xt_options* opt,
                      xt_tracker** out) {
  g_err.clear();
  if (!out) return fail(XT_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!table || !ref) return fail(XT_ERR_INVALID, "table or reference is null");
  if (n < 1 || n > (1 << 24)) return fail(XT_ERR_INVALID, "n_elements must be in 1..2^24");
  if (!(ref->mass0 > 0.0) || !(ref->p0c > 0.0) || !(ref->q0 == ref->q0))
    return fail(XT_ERR_INVALID, "reference needs mass0 > 0 and p0c > 0");
  xt_options o;
  xt_options_default(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  std::unique_ptr<xt_tracker> t(new xt_tracker());
  t->opt = o;
  t->rc = ref_constants(*ref);
  t->ref = {t->rc.beta0, t->rc.gamma0, t->rc.bg0, t->rc.ib0, t->rc.twoib0, t->rc.p0c, t->rc.uc15, t->rc.ig02,
            1.0 / t->rc.p0c};
  t->sn = sin_table();
  std::string err;
  rc = compile_lattice(table, n, t->rc, &t->lat, &err);
  if (rc) return fail(rc, err);
  t->table.assign(table, table + n);
  CK(cudaGetDevice(&t->device));
  int e = device_sm_count(&t->sm_count);
  if (e) return cuda_fail((cudaError_t)e, "device attribute");
  e = device_smem_optin(&t->smem_max);
  if (e) return cuda_fail((cudaError_t)e, "device attribute");
  {
    double tab[XT_SPECIAL_N];
    special_table(tab);
    e = upload_special_table(tab);
    if (e) return cuda_fail((cudaError_t)e, "beam-beam constant table");
  }
  rc = dev_alloc(&t->d_lat, t->lat.bytes.size());
  if (rc) return rc;
  if (!t->lat.bytes.empty())
    CK(cudaMemcpy(t->d_lat, t->lat.bytes.data(), t->lat.bytes.size(), cudaMemcpyHostToDevice));
  std::vector<double> xi, F;
  std::vector<int32_t> guide;
  photon_table(&xi, &F, &guide);
  t->spec_k = (int)xi.size();
  for (int j = 0; j < XT_EXPNEG_N; j++) xi.push_back(std::exp(-(double)j / 64.0));
  rc = dev_alloc(&t->d_spec_xi, xi.size());
  if (rc) return rc;
  rc = dev_alloc(&t->d_spec_F, F.size());
  if (rc) return rc;
  rc = dev_alloc(&t->d_spec_guide, guide.size());
  if (rc) return rc;
  CK(cudaMemcpy(t->d_spec_xi, xi.data(), xi.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(t->d_spec_F, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(t->d_spec_guide, guide.data(), guide.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  rc = dev_alloc(&t->d_scal, 8);
  if (rc) return rc;
  CK(cudaMemset(t->d_scal, 0, 8 * sizeof(int32_t)));
  CK(cudaHostAlloc((void**)&t->h_cancel, sizeof(int32_t), cudaHostAllocMapped));
  *t->h_cancel = 0;
  CK(cudaHostGetDevicePointer((void**)&t->d_cancel, t->h_cancel, 0));
  rc = build_device_chunks(t.get(), eff_chunk(t.get()));
  if (rc) return rc;
  *out = t.release();
  return XT_OK;
}

void xt_tracker_destroy(xt_tracker* t) {
  if (!t) return;
  cudaDeviceSynchronize();
  evict_plans_of(t);
  cudaFree(t->d_lat);
  cudaFree(t->d_chunks);
  cudaFree(t->d_spec_xi);
  cudaFree(t->d_spec_F);
  cudaFree(t->d_spec_guide);
  cudaFree(t->d_scal);
  cudaFree(t->d_idx);
  cudaFree(t->d_counts);
  cudaFree(t->d_stage);
  cudaFree(t->d_refine);
  cudaFree(t->d_rowoff);
  if (t->h_cancel) cudaFreeHost(t->h_cancel);
  for (auto& pr : t->ev) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  delete t;
}

int xt_tracker_set_options(xt_tracker* t, const xt_options* o) {
  g_err.clear();
  if (!t || !o) return fail(XT_ERR_INVALID, "null argument");
  int rc = check_options(*o);
  if (rc) return rc;
  t->opt = *o;
  return build_device_chunks(t, eff_chunk(t));
}

int xt_tracker_get_options(const xt_tracker* t, xt_options* o) {
  if (!t || !o) return fail(XT_ERR_INVALID, "null argument");
  *o = t->opt;
  return XT_OK;
}

int xt_track(xt_tracker* t, const xt_particles* p, int64_t start_turn, int64_t n_turns, void* stream) {
  g_err.clear();
  if (!t) return fail(XT_ERR_INVALID, "tracker is null");
  if (!particles_ok(p)) return fail(XT_ERR_INVALID, "particle arrays are null or n out of range");
  if (start_turn < 0 || n_turns < 0 || start_turn + n_turns > 0x7fffffff)
    return fail(XT_ERR_INVALID, "turn range outside 0..2^31-1");
  return track_device(t, p, start_turn, n_turns, stream);
}

int xt_track_host(xt_tracker* t, const xt_particles* h, int64_t start_turn, int64_t n_turns, void* stream) {
  g_err.clear();
  if (!t) return fail(XT_ERR_INVALID, "tracker is null");
  if (!particles_ok(h)) return fail(XT_ERR_INVALID, "particle arrays are null or n out of range");
  if (start_turn < 0 || n_turns < 0 || start_turn + n_turns > 0x7fffffff)
    return fail(XT_ERR_INVALID, "turn range outside 0..2^31-1");
  const int64_t n = h->n;
  if (n == 0) return XT_OK;
  // 9 doubles + 3 int32 + 1 int64 per particle, each array 256-byte aligned
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bd = al(n * 8), bi = al(n * 4);
  if (n > t->stage_n) {
    cudaFree(t->d_stage);
    t->d_stage = nullptr;
    t->stage_n = -1;
    cudaError_t e = cudaMalloc(&t->d_stage, 10 * bd + 3 * bi);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc staging");
    t->stage_n = n;
  }
  uint8_t* base = (uint8_t*)t->d_stage;
  xt_particles d;
  double** fd[9] = {&d.x, &d.px, &d.y, &d.py, &d.zeta, &d.delta, &d.ptau, &d.rpp, &d.rvv};
  double* const hd[9] = {h->x, h->px, h->y, h->py, h->zeta, h->delta, h->ptau, h->rpp, h->rvv};
  for (int k = 0; k < 9; k++) *fd[k] = (double*)(base + k * bd);
  d.state = (int32_t*)(base + 9 * bd);
  d.at_turn = (int32_t*)(base + 9 * bd + bi);
  d.at_element = (int32_t*)(base + 9 * bd + 2 * bi);
  d.particle_id = (const int64_t*)(base + 9 * bd + 3 * bi);
  d.n = n;
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < 9; k++) CK(cudaMemcpyAsync(*fd[k], hd[k], n * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d.state, h->state, n * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d.at_turn, h->at_turn, n * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d.at_element, h->at_element, n * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync((void*)d.particle_id, h->particle_id, n * 8, cudaMemcpyHostToDevice, s));
  int rc = track_device(t, &d, start_turn, n_turns, stream);
  if (rc) return rc;
  for (int k = 0; k < 9; k++) CK(cudaMemcpyAsync(hd[k], *fd[k], n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->state, d.state, n * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->at_turn, d.at_turn, n * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->at_element, d.at_element, n * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return XT_OK;
}

int xt_sync_status(xt_tracker* t, void* stream) {
  g_err.clear();
  if (!t) return fail(XT_ERR_INVALID, "tracker is null");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t st = 0;
  CK(cudaMemcpyAsync(&st, t->d_scal, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaMemsetAsync(t->d_scal, 0, sizeof(int32_t), s));
  CK(cudaStreamSynchronize(s));
  if (st == XT_ERR_TIMEOUT) return fail(st, "cycle budget exceeded; tracking stopped at a turn boundary");
  if (st == XT_ERR_CANCELLED) return fail(st, "tracking cancelled at a turn boundary");
  if (st != 0) return fail(XT_ERR_CUDA, "lattice staging did not complete");
  return XT_OK;
}

int xt_cancel(xt_tracker* t) {
  if (!t) return fail(XT_ERR_INVALID, "tracker is null");
  __atomic_store_n(t->h_cancel, 1, __ATOMIC_SEQ_CST);
  return XT_OK;
}

int xt_reset_cancel(xt_tracker* t) {
  if (!t) return fail(XT_ERR_INVALID, "tracker is null");
  __atomic_store_n(t->h_cancel, 0, __ATOMIC_SEQ_CST);
  return XT_OK;
}

int xt_set_profiling(xt_tracker* t, int enable) {
  g_err.clear();
  if (!t) return fail(XT_ERR_INVALID, "tracker is null");
  t->prof = enable != 0;
  t->ev_used = 0;
  return XT_OK;
}

int xt_kernel_time(xt_tracker* t, double* total_ms, int64_t* launches) {
  g_err.clear();
  if (!t || !total_ms || !launches) return fail(XT_ERR_INVALID, "null argument");
  double sum = 0.0;
  for (size_t i = 0; i < t->ev_used; i++) {
    CK(cudaEventSynchronize(t->ev[i].second));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t->ev[i].first, t->ev[i].second));
    sum += ms;
  }
  *total_ms = sum;
  *launches = (int64_t)t->ev_used;
  t->ev_used = 0;
  return XT_OK;
}

int xt_fp64_peak(double* flops_per_s, double* elapsed_ms, void* stream) {
  g_err.clear();
  if (!flops_per_s || !elapsed_ms) return fail(XT_ERR_INVALID, "null argument");
  int sms = 0;
  int e = device_sm_count(&sms);
  if (e) return cuda_fail((cudaError_t)e, "device attribute");
  // every probe variant at 4, 8 and 16 blocks of 128 threads per SM; the
  // fastest is the measured ceiling
  const int block = 128, iters = 8192;
  const int max_grid = sms * 16;
  double* buf = nullptr;
  int rc = dev_alloc(&buf, (size_t)max_grid * block);
  if (rc) return rc;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t ce = cudaEventCreate(&a);
  if (ce == cudaSuccess) ce = cudaEventCreate(&b);
  cudaStream_t s = (cudaStream_t)stream;
  double best = 0.0, best_ms = 0.0;
  for (int variant = 0; variant < 4 && ce == cudaSuccess; variant++) {
    for (int per_sm : {4, 8, 16}) {
      const int grid = sms * per_sm;
      int chains = 0;
      e = launch_fp64_probe(buf, grid, block, 64, variant, &chains, stream);  // warm-up
      if (e) { ce = (cudaError_t)e; break; }
      if ((ce = cudaEventRecord(a, s)) != cudaSuccess) break;
      e = launch_fp64_probe(buf, grid, block, iters, variant, &chains, stream);
      if (e) { ce = (cudaError_t)e; break; }
      if ((ce = cudaEventRecord(b, s)) != cudaSuccess) break;
      if ((ce = cudaEventSynchronize(b)) != cudaSuccess) break;
      float ms = 0.f;
      if ((ce = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) break;
      // chains independent fmas per thread per iteration, 2 flops each
      const double f = 2.0 * chains * (double)iters * (double)grid * (double)block / (ms * 1e-3);
      if (f > best) { best = f; best_ms = ms; }
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaStreamSynchronize(s);
  cudaFree(buf);
  if (ce != cudaSuccess) return cuda_fail(ce, "fp64 probe");
  *flops_per_s = best;
  *elapsed_ms = best_ms;
  return XT_OK;
}

// Loss-location refinement tables (see xt_refine_losses in xtgb.h): entrance
// position and reference frame of every row, record offsets, previous
// aperture, and the laboratory-frame polygon of every aperture from rays at
// n_angles angles about its frame origin.
static bool is_aperture_type(int t) {
  return t == XT_APERTURE || t == XT_APERTURE_RECT || t == XT_APERTURE_ELLIPSE;
}

// distance from the aperture's frame origin to its boundary along angle phi;
// negative if the origin is not strictly inside
static double boundary_distance(const xt_element& e, double phi) {
  const double c = std::cos(phi), s = std::sin(phi);
  if (e.type == XT_APERTURE) return e.p[0];
  if (e.type == XT_APERTURE_ELLIPSE) {
    const double a = e.p[0], b = e.p[1];
    return 1.0 / std::sqrt(c * c / (a * a) + s * s / (b * b));
  }
  const double x0 = e.p[0], x1 = e.p[1], y0 = e.p[2], y1 = e.p[3];
  if (!(x0 < 0.0 && 0.0 < x1 && y0 < 0.0 && 0.0 < y1)) return -1.0;
  double t = INFINITY;
  if (c > 0.0) t = std::min(t, x1 / c);
  if (c < 0.0) t = std::min(t, x0 / c);
  if (s > 0.0) t = std::min(t, y1 / s);
  if (s < 0.0) t = std::min(t, y0 / s);
  return t;
}

static int build_refine_tables(xt_tracker* t, int n_angles) {
  const int64_t n = t->lat.n_el;
  std::vector<int32_t> row_off(n, -1), prev(n, -1), pidx(n, -1);
  std::vector<double> spos(n + 1, 0.0), frame(4 * n, 0.0);
  double th = 0.0, fdx = 0.0, fdy = 0.0;
  int64_t last = -1;
  for (int64_t i = 0; i < n; i++) {
    const xt_element& e = t->table[i];
    row_off[i] = t->lat.row_rec[(size_t)i];
    frame[4 * i] = std::cos(th);
    frame[4 * i + 1] = std::sin(th);
    frame[4 * i + 2] = fdx;
    frame[4 * i + 3] = fdy;
    spos[i + 1] = spos[i] + (e.type == XT_DRIFT ? e.p[0]
                             : (e.type == XT_QUAD ? e.p[1] : (e.type == XT_BEND ? e.p[2] : 0.0)));
    if (e.type == XT_XYSHIFT) {
      const double c = std::cos(th), sn = std::sin(th);
      fdx = fdx + (c * e.p[0] - sn * e.p[1]);
      fdy = fdy + (sn * e.p[0] + c * e.p[1]);
    } else if (e.type == XT_SROTATION) {
      th = th + e.p[0];
    }
    if (is_aperture_type(e.type)) last = i;
  }
  if (last < 0) return fail(XT_ERR_INVALID, "refinement needs an aperture row in the table");
  const double two_pi = 6.283185307179586;
  std::vector<double> polys;
  int32_t np = 0;
  for (int64_t i = 0; i < n; i++) {
    const xt_element& e = t->table[i];
    if (!is_aperture_type(e.type)) continue;
    prev[i] = (int32_t)last;
    last = i;
    const double c = frame[4 * i], sn = frame[4 * i + 1];
    std::vector<double> v(2 * (size_t)n_angles);
    bool ok = true;
    for (int kk = 0; kk < n_angles; kk++) {
      const double phi = two_pi * (double)kk / (double)n_angles;
      const double r = boundary_distance(e, phi);
      if (!(r > 0.0)) ok = false;
      const double lx = r * std::cos(phi), ly = r * std::sin(phi);
      v[2 * kk] = (c * lx - sn * ly) + frame[4 * i + 2];
      v[2 * kk + 1] = (sn * lx + c * ly) + frame[4 * i + 3];
    }
    if (!ok) continue;
    pidx[i] = np++;
    polys.insert(polys.end(), v.begin(), v.end());
  }
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_off = al(n * 4), b_prev = al(n * 4), b_pidx = al(n * 4), b_spos = al((n + 1) * 8),
               b_frame = al(4 * n * 8), b_poly = al(std::max<size_t>(polys.size(), 1) * 8);
  const size_t total = b_off + b_prev + b_pidx + b_spos + b_frame + b_poly;
  std::vector<uint8_t> h(total, 0);
  size_t o = 0;
  std::memcpy(h.data() + o, row_off.data(), n * 4);
  const size_t o_off = o;
  o += b_off;
  std::memcpy(h.data() + o, prev.data(), n * 4);
  const size_t o_prev = o;
  o += b_prev;
  std::memcpy(h.data() + o, pidx.data(), n * 4);
  const size_t o_pidx = o;
  o += b_pidx;
  std::memcpy(h.data() + o, spos.data(), (n + 1) * 8);
  const size_t o_spos = o;
  o += b_spos;
  std::memcpy(h.data() + o, frame.data(), 4 * n * 8);
  const size_t o_frame = o;
  o += b_frame;
  if (!polys.empty()) std::memcpy(h.data() + o, polys.data(), polys.size() * 8);
  const size_t o_poly = o;
  if (t->d_refine) cudaFree(t->d_refine);
  t->d_refine = nullptr;
  t->refine_angles = 0;
  int rc = dev_alloc(&t->d_refine, total);
  if (rc) return rc;
  CK(cudaMemcpy(t->d_refine, h.data(), total, cudaMemcpyHostToDevice));
  RefineArgs& a = t->refine_tab;
  std::memset(&a, 0, sizeof(a));
  a.lat = t->d_lat;
  a.row_off = (const int32_t*)(t->d_refine + o_off);
  a.prev_ap = (const int32_t*)(t->d_refine + o_prev);
  a.poly_idx = (const int32_t*)(t->d_refine + o_pidx);
  a.spos = (const double*)(t->d_refine + o_spos);
  a.frame = (const double*)(t->d_refine + o_frame);
  a.polys = (const double*)(t->d_refine + o_poly);
  a.n_el = (int32_t)n;
  a.n_angles = n_angles;
  a.ref = t->ref;
  a.sn = t->sn;
  t->refine_angles = n_angles;
  return XT_OK;
}

int xt_refine_losses(xt_tracker* t, const xt_particles* p, double ds, int32_t n_angles, double* s_loss,
                     void* stream) {
  g_err.clear();
  if (!t || !particles_ok(p) || !s_loss) return fail(XT_ERR_INVALID, "null tracker, particles or s_loss");
  if (!(ds > 0.0) || n_angles < 8 || n_angles > 1024)
    return fail(XT_ERR_INVALID, "refinement needs ds > 0 and 8 <= n_angles <= 1024");
  if (t->refine_angles != n_angles) {
    int rc = build_refine_tables(t, n_angles);
    if (rc) return rc;
  }
  if (p->n == 0) return XT_OK;
  RefineArgs a = t->refine_tab;
  a.ds = ds;
  a.x = p->x; a.px = p->px; a.y = p->y; a.py = p->py; a.zeta = p->zeta;
  a.delta = p->delta; a.ptau = p->ptau; a.rpp = p->rpp; a.rvv = p->rvv;
  a.state = p->state;
  a.at_element = p->at_element;
  a.s_loss = s_loss;
  a.n = p->n;
  int e = launch_refine(a, stream);
  if (e) return cuda_fail((cudaError_t)e, "refinement launch");
  return XT_OK;
}

int xt_track_monitor(xt_tracker* t, const xt_particles* p, int64_t turn, double* out, void* stream) {
  g_err.clear();
  if (!t || !particles_ok(p) || !out) return fail(XT_ERR_INVALID, "null tracker, particles or out");
  if (turn < 0 || turn > 0x7ffffffe) return fail(XT_ERR_INVALID, "turn outside 0..2^31-2");
  if (p->n > XT_MONITOR_MAX_PARTICLES) return fail(XT_ERR_INVALID, "the monitor takes at most 4096 particles");
  const int64_t n_el = t->lat.n_el;
  if (!t->d_rowoff) {
    int rc = dev_alloc(&t->d_rowoff, (size_t)n_el);
    if (rc) return rc;
    CK(cudaMemcpy(t->d_rowoff, t->lat.row_rec.data(), (size_t)n_el * 4, cudaMemcpyHostToDevice));
  }
  if (p->n == 0) return XT_OK;
  MonitorArgs a;
  std::memset(&a, 0, sizeof(a));
  a.lat = t->d_lat;
  a.row_off = t->d_rowoff;
  a.n_el = (int32_t)n_el;
  a.turn = (int32_t)turn;
  a.n = p->n;
  a.x = p->x; a.px = p->px; a.y = p->y; a.py = p->py; a.zeta = p->zeta;
  a.delta = p->delta; a.ptau = p->ptau; a.rpp = p->rpp; a.rvv = p->rvv;
  a.state = p->state; a.at_turn = p->at_turn; a.at_element = p->at_element;
  a.pid = p->particle_id;
  a.out = out;
  a.seed = t->opt.seed;
  a.spec_xi = t->d_spec_xi;
  a.spec_F = t->d_spec_F;
  a.spec_guide = t->d_spec_guide;
  a.spec_k = t->spec_k;
  a.ref = t->ref;
  a.sn = t->sn;
  int e = launch_monitor(a, t->opt.radiation, stream);
  if (e) return cuda_fail((cudaError_t)e, "monitor launch");
  return XT_OK;
}

int xt_element_flops(const xt_tracker* t, int64_t* out, int64_t n) {
  if (!t || !out || n != t->lat.n_el) return fail(XT_ERR_INVALID, "need an array of n_elements entries");
  for (int64_t i = 0; i < n; i++) out[i] = flops_of_row(t->table[i], t->opt.radiation);
  return XT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch parameters for xt_track_noalloc (xt_noalloc.cu).  Uses the tracker's
// existing chunk table as built at create/set_options time; no allocation.
namespace xt {
void set_error(const std::string& msg) { g_err = msg; }

int noalloc_prepare(xt_tracker* t, const xt_particles* p, int64_t n_turns, TrackArgs* a, int* block,
                    int* grid, size_t* smem, int* seg, int* rad) {
  if (!t->d_chunks) return fail(XT_ERR_INVALID, "tracker has no lattice chunk table");
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != t->device)
    return fail(XT_ERR_INVALID, "xt_track_noalloc: the current device (" + std::to_string(dev) +
                                    ") is not the tracker's (" + std::to_string(t->device) + ")");
  *block = eff_block(t);
  *smem = track_smem_bytes(*block, t->chunk_built, kind_of(t));
  int rc = grid_for(t, *block, *smem, grid);
  if (rc) return rc;
  *seg = eff_segment(t, p->n, n_turns);
  *rad = kind_of(t);
  fill_args(t, p, a);
  return XT_OK;
}
}  // namespace xt

// ---------------------------------------------------------------------------
// Autotuner: block x chunk x segment on a probe copy of the particles.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<uint64_t, int64_t, int>, std::tuple<int, int, int>> g_tune_cache;
}  // namespace

extern "C" int xt_autotune(xt_tracker* t, const xt_particles* probe, int64_t probe_turns, void* stream) {
  g_err.clear();
  if (!t || !particles_ok(probe) || probe->n == 0 || probe_turns < 1)
    return fail(XT_ERR_INVALID, "autotune needs a tracker, probe particles and probe_turns >= 1");
  const auto key = std::make_tuple(t->lat.hash, probe->n, t->opt.radiation);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      xt_options o = t->opt;
      o.block = std::get<0>(it->second);
      o.chunk_bytes = std::get<1>(it->second);
      o.segment_turns = std::get<2>(it->second);
      return xt_tracker_set_options(t, &o);
    }
  }
  const int64_t n = probe->n;
  cudaStream_t s = (cudaStream_t)stream;
  // scratch copy of the probe (13 arrays) and two events, released on every
  // return path (after the stream has finished with them)
  struct Scratch {
    cudaStream_t s;
    uint8_t* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch() {
      cudaStreamSynchronize(s);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (buf) cudaFree(buf);
    }
  } sc{s};
  const size_t bd = ((size_t)n * 8 + 255) & ~(size_t)255, bi = ((size_t)n * 4 + 255) & ~(size_t)255;
  CK(cudaMalloc((void**)&sc.buf, 10 * bd + 3 * bi));
  uint8_t* const buf = sc.buf;
  xt_particles w;
  double** fd[9] = {&w.x, &w.px, &w.y, &w.py, &w.zeta, &w.delta, &w.ptau, &w.rpp, &w.rvv};
  double* const src[9] = {probe->x, probe->px, probe->y, probe->py, probe->zeta,
                          probe->delta, probe->ptau, probe->rpp, probe->rvv};
  for (int k = 0; k < 9; k++) *fd[k] = (double*)(buf + k * bd);
  w.state = (int32_t*)(buf + 9 * bd);
  w.at_turn = (int32_t*)(buf + 9 * bd + bi);
  w.at_element = (int32_t*)(buf + 9 * bd + 2 * bi);
  w.particle_id = probe->particle_id;
  w.n = n;
  auto restore = [&]() -> int {
    for (int k = 0; k < 9; k++) CK(cudaMemcpyAsync(*fd[k], src[k], n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.state, probe->state, n * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.at_turn, probe->at_turn, n * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(w.at_element, probe->at_element, n * 4, cudaMemcpyDeviceToDevice, s));
    return XT_OK;
  };
  const xt_options saved = t->opt;
  CK(cudaEventCreate(&sc.e0));
  CK(cudaEventCreate(&sc.e1));
  const cudaEvent_t e0 = sc.e0, e1 = sc.e1;
  // a CUDA error inside the search sets rc and leaves the loops
#define TUNE_CK(call)                                  \
  {                                                    \
    const cudaError_t _e = (call);                     \
    if (_e != cudaSuccess) {                           \
      rc = cuda_fail(_e, #call);                       \
      break;                                           \
    }                                                  \
  }
  float best = 1e30f;
  int bb = DEFAULT_BLOCK, bc = DEFAULT_CHUNK, bs = 0;
  const int blocks[] = {64, 128, 256};
  const int chunks[] = {2048, 4096, 8192, 16384};
  const int segs[] = {0, 1, 4};
  int rc = XT_OK;
  for (int blk : blocks) {
    for (int ch : chunks) {
      for (int sg : segs) {
        if (sg > probe_turns) continue;
        xt_options o = saved;
        o.block = blk;
        o.chunk_bytes = ch;
        o.segment_turns = sg;
        if (xt_tracker_set_options(t, &o) != XT_OK) continue;
        int bps = 0;
        const size_t sm = track_smem_bytes(blk, t->chunk_built, kind_of(t));
        if (sm > (size_t)t->smem_max || track_occupancy(o.radiation + (t->lat.thick ? 3 : 0), blk, sm, &bps) || bps < 1) continue;
        if ((rc = restore())) break;
        TUNE_CK(cudaEventRecord(e0, s));
        rc = track_device(t, &w, 0, probe_turns, stream);
        if (rc) break;
        TUNE_CK(cudaEventRecord(e1, s));
        TUNE_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        TUNE_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; bb = blk; bc = ch; bs = sg; }
      }
      if (rc) break;
    }
    if (rc) break;
  }
#undef TUNE_CK
  if (rc) { t->opt = saved; build_device_chunks(t, eff_chunk(t)); return rc; }
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = std::make_tuple(bb, bc, bs);
  }
  xt_options o = saved;
  o.block = bb;
  o.chunk_bytes = bc;
  o.segment_turns = bs;
  return xt_tracker_set_options(t, &o);
}

// ---------------------------------------------------------------------------
// Batched seeds.
namespace {

struct BatchPlan {
  int device = 0;
  int n_seeds = 0;
  int64_t max_n = 0;
  SeedDev* d_seeds = nullptr;
  int32_t* d_order = nullptr;
  int64_t* d_idx_base = nullptr;
  int64_t* d_prefix = nullptr;
  int32_t* d_idx = nullptr;
  int32_t* d_counts = nullptr;
  int32_t* d_n_alive = nullptr;
  int32_t* d_scal = nullptr;  // [0] status [1] tile counter [2] turn base
  std::vector<const xt_tracker*> trackers;  // the seeds' trackers, for eviction on destroy
  // captured graphs, keyed by every value the captured launches bake in
  std::map<std::vector<uint64_t>, cudaGraphExec_t> graphs;
  ~BatchPlan() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    cudaFree(d_seeds); cudaFree(d_order); cudaFree(d_idx_base); cudaFree(d_prefix);
    cudaFree(d_idx); cudaFree(d_counts); cudaFree(d_n_alive); cudaFree(d_scal);
  }
};

std::mutex g_plan_mu;

// A plan bakes in every device pointer of every seed (lattice, chunk table,
// all particle arrays) and the counts, so all of them are part of its key:
// a call with any buffer replaced gets a plan of its own.
std::vector<uintptr_t> plan_key(xt_tracker* const* trs, const xt_particles* ps, int32_t ns) {
  std::vector<uintptr_t> key;
  for (int i = 0; i < ns; i++) {
    const xt_tracker* t = trs[i];
    const xt_particles& p = ps[i];
    key.push_back((uintptr_t)t);
    key.push_back(t ? (uintptr_t)t->d_lat : 0);
    key.push_back(t ? (uintptr_t)t->d_chunks : 0);
    key.push_back(t ? (uintptr_t)t->n_chunks : 0);
    key.push_back(t ? (uintptr_t)t->chunk_built : 0);
    for (const void* a : {(const void*)p.x, (const void*)p.px, (const void*)p.y, (const void*)p.py,
                          (const void*)p.zeta, (const void*)p.delta, (const void*)p.ptau, (const void*)p.rpp,
                          (const void*)p.rvv, (const void*)p.state, (const void*)p.at_turn,
                          (const void*)p.at_element, (const void*)p.particle_id})
      key.push_back((uintptr_t)a);
    key.push_back((uintptr_t)p.n);
  }
  return key;
}
std::map<std::vector<uintptr_t>, std::unique_ptr<BatchPlan>> g_plans;

int make_plan(xt_tracker* const* trs, const xt_particles* ps, int32_t ns, BatchPlan* pl) {
  std::vector<SeedDev> sd(ns);
  std::vector<int64_t> base(ns);
  int64_t tot = 0;
  pl->max_n = 0;
  for (int i = 0; i < ns; i++) {
    const xt_tracker* t = trs[i];
    const xt_particles* p = &ps[i];
    SeedDev& d = sd[i];
    d.lat = t->d_lat; d.chunks = t->d_chunks; d.n_chunks = t->n_chunks; d.n_el = (int32_t)t->lat.n_el;
    d.x = p->x; d.px = p->px; d.y = p->y; d.py = p->py; d.zeta = p->zeta; d.delta = p->delta;
    d.ptau = p->ptau; d.rpp = p->rpp; d.rvv = p->rvv; d.state = p->state; d.at_turn = p->at_turn;
    d.at_element = p->at_element; d.pid = p->particle_id; d.n = p->n;
    base[i] = tot;
    tot += p->n;
    pl->max_n = std::max(pl->max_n, p->n);
  }
  std::vector<int32_t> order(ns);
  for (int i = 0; i < ns; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ps[a].n > ps[b].n; });
  pl->n_seeds = ns;
  pl->trackers.assign(trs, trs + ns);
  int rc;
  if ((rc = dev_alloc(&pl->d_seeds, ns))) return rc;
  if ((rc = dev_alloc(&pl->d_order, ns))) return rc;
  if ((rc = dev_alloc(&pl->d_idx_base, ns))) return rc;
  if ((rc = dev_alloc(&pl->d_prefix, ns + 1))) return rc;
  if ((rc = dev_alloc(&pl->d_idx, (size_t)tot))) return rc;
  const int64_t bps = (pl->max_n + 1023) / 1024;
  if ((rc = dev_alloc(&pl->d_counts, (size_t)(bps * ns + 1)))) return rc;
  if ((rc = dev_alloc(&pl->d_n_alive, ns))) return rc;
  if ((rc = dev_alloc(&pl->d_scal, 4))) return rc;
  CK(cudaMemcpy(pl->d_seeds, sd.data(), ns * sizeof(SeedDev), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pl->d_order, order.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pl->d_idx_base, base.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice));
  CK(cudaMemset(pl->d_scal, 0, 4 * sizeof(int32_t)));
  return XT_OK;
}

int enqueue_batched(xt_tracker* t0, BatchPlan* pl, int kind, int64_t n_turns, int seg, int block, size_t smem,
                    int grid, void* stream) {
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.seeds = pl->d_seeds;
  a.seed_order = pl->d_order;
  a.tile_prefix = pl->d_prefix;
  a.idx = pl->d_idx;
  a.idx_base = pl->d_idx_base;
  a.n_alive = pl->d_n_alive;
  a.tile_counter = pl->d_scal + 1;
  a.status = pl->d_scal;
  a.cancel = t0->d_cancel;
  a.turn_base = pl->d_scal + 2;
  a.n_seeds = pl->n_seeds;
  a.chunk_bytes = t0->chunk_built;
  a.max_cycles = t0->opt.max_cycles;
  a.seed = t0->opt.seed;
  a.spec_xi = t0->d_spec_xi;
  a.spec_F = t0->d_spec_F;
  a.spec_guide = t0->d_spec_guide;
  a.spec_k = t0->spec_k;
  a.ref = t0->ref;
  a.sn = t0->sn;
  for (int64_t done = 0; done < n_turns; done += seg) {
    const int nt = (int)std::min<int64_t>(seg, n_turns - done);
    int e = launch_compact_batched(pl->d_seeds, pl->n_seeds, pl->d_idx_base, pl->d_idx, pl->d_n_alive,
                                   pl->d_counts, pl->max_n, stream);
    if (e) return cuda_fail((cudaError_t)e, "batched compaction");
    e = launch_tile_prefix(pl->d_n_alive, pl->d_order, pl->n_seeds, pl->d_prefix, pl->d_scal + 1, stream);
    if (e) return cuda_fail((cudaError_t)e, "tile prefix");
    a.turn_off = (int32_t)done;
    a.n_turns = nt;
    e = launch_track_batched(a, kind, block, grid, smem, stream);
    if (e) return cuda_fail((cudaError_t)e, "batched tracking launch");
  }
  return XT_OK;
}

}  // namespace

extern "C" int xt_track_batched(xt_tracker* const* trs, const xt_particles* ps, int32_t ns, int64_t start_turn,
                                int64_t n_turns, int32_t graph, void* stream) {
  g_err.clear();
  if (!trs || !ps || ns < 1) return fail(XT_ERR_INVALID, "need at least one seed");
  if (start_turn < 0 || n_turns < 0 || start_turn + n_turns > 0x7fffffff)
    return fail(XT_ERR_INVALID, "turn range outside 0..2^31-1");
  xt_tracker* t0 = trs[0];
  if (!t0) return fail(XT_ERR_INVALID, "tracker is null");
  int64_t total = 0;
  for (int i = 0; i < ns; i++) {
    const xt_tracker* t = trs[i];
    if (!t || !particles_ok(&ps[i])) return fail(XT_ERR_INVALID, "seed " + std::to_string(i) + ": bad tracker or particles");
    if (t->device != t0->device || t->opt.radiation != t0->opt.radiation ||
        std::memcmp(&t->ref, &t0->ref, sizeof(RefDev)) != 0)
      return fail(XT_ERR_INVALID, "all seeds need the same device, reference and radiation mode");
    total += ps[i].n;
  }
  if (total > 0x7fffffff) return fail(XT_ERR_INVALID, "too many particles in the batch");
  if (n_turns == 0 || total == 0) return XT_OK;
  bool thick = false;
  for (int i = 0; i < ns; i++) thick = thick || trs[i]->lat.thick;
  const int kind = t0->opt.radiation + (thick ? 3 : 0);
  const int block = eff_block(t0);
  const int chunk = eff_chunk(t0);
  for (int i = 0; i < ns; i++) {
    int rc = build_device_chunks(trs[i], chunk);
    if (rc) return rc;
  }
  const size_t smem = track_smem_bytes(block, chunk, kind);
  if (smem > (size_t)t0->smem_max)
    return fail(XT_ERR_INVALID, "block x 2 x chunk_bytes exceeds the shared memory of one block");
  int bpsm = 0;
  int e = batched_occupancy(kind, block, smem, &bpsm);
  if (e) return cuda_fail((cudaError_t)e, "occupancy");
  if (bpsm < 1) return fail(XT_ERR_INVALID, "launch configuration does not fit on an SM");
  const int grid = bpsm * t0->sm_count;
  // plan keyed by the tracker, chunk-table and particle pointers
  std::vector<uintptr_t> key = plan_key(trs, ps, ns);
  std::lock_guard<std::mutex> g(g_plan_mu);
  auto it = g_plans.find(key);
  if (it == g_plans.end()) {
    std::unique_ptr<BatchPlan> pl(new BatchPlan());
    int rc = make_plan(trs, ps, ns, pl.get());
    if (rc) return rc;
    it = g_plans.emplace(key, std::move(pl)).first;
  }
  BatchPlan* pl = it->second.get();
  const int seg = eff_segment(t0, total / ns, n_turns);
  e = launch_set_int(pl->d_scal + 2, (int32_t)start_turn, stream);
  if (e) return cuda_fail((cudaError_t)e, "turn base");
  if (!graph) return enqueue_batched(t0, pl, kind, n_turns, seg, block, smem, grid, stream);
  // the graph's key: the launch shape and every field of t0 that
  // enqueue_batched copies into the kernel arguments (seed, cycle budget,
  // cancel flag, spectrum tables, reference constants, sine table)
  std::vector<uint64_t> gk = {(uint64_t)n_turns, (uint64_t)seg, (uint64_t)block, (uint64_t)chunk, (uint64_t)kind,
                              (uint64_t)grid, (uint64_t)smem, t0->opt.seed, (uint64_t)t0->opt.max_cycles,
                              (uint64_t)(uintptr_t)t0->d_cancel, (uint64_t)(uintptr_t)t0->d_spec_xi,
                              (uint64_t)(uintptr_t)t0->d_spec_F, (uint64_t)(uintptr_t)t0->d_spec_guide,
                              (uint64_t)t0->spec_k, (uint64_t)t0->chunk_built};
  auto push_bytes = [&gk](const void* v, size_t nb) {
    for (size_t o = 0; o < nb; o += 8) {
      uint64_t w = 0;
      std::memcpy(&w, (const uint8_t*)v + o, std::min<size_t>(8, nb - o));
      gk.push_back(w);
    }
  };
  push_bytes(&t0->ref, sizeof(t0->ref));
  push_bytes(&t0->sn, sizeof(t0->sn));
  auto gi = pl->graphs.find(gk);
  if (gi == pl->graphs.end()) {
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    // make sure kernel attributes are set before capture
    int dummy = 0;
    batched_occupancy(kind, block, smem, &dummy);
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_batched(t0, pl, kind, n_turns, seg, block, smem, grid, cs);
    cudaGraph_t gr;
    cudaError_t ce = cudaStreamEndCapture(cs, &gr);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (ce != cudaSuccess) return cuda_fail(ce, "graph capture");
    cudaGraphExec_t ex;
    ce = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
    gi = pl->graphs.emplace(gk, ex).first;
  }
  CK(cudaGraphLaunch(gi->second, (cudaStream_t)stream));
  return XT_OK;
}

extern "C" int xt_batched_sync_status(xt_tracker* const* trs, const xt_particles* ps, int32_t ns, void* stream) {
  g_err.clear();
  if (!trs || !ps || ns < 1) return fail(XT_ERR_INVALID, "need at least one seed");
  std::vector<uintptr_t> key = plan_key(trs, ps, ns);
  std::lock_guard<std::mutex> g(g_plan_mu);
  auto it = g_plans.find(key);
  if (it == g_plans.end()) return fail(XT_ERR_INVALID, "no batched launch with these arguments");
  int32_t st = 0;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(&st, it->second->d_scal, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaMemsetAsync(it->second->d_scal, 0, sizeof(int32_t), s));
  CK(cudaStreamSynchronize(s));
  return st;
}

// Frees every batched plan that names tracker t (called by
// xt_tracker_destroy, after the device has finished its work).
void evict_plans_of(const xt_tracker* t) {
  std::lock_guard<std::mutex> g(g_plan_mu);
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    const auto& trs = it->second->trackers;
    if (std::find(trs.begin(), trs.end(), t) != trs.end())
      it = g_plans.erase(it);
    else
      ++it;
  }
}

extern "C" void xt_batched_release(void) {
  std::lock_guard<std::mutex> g(g_plan_mu);
  cudaDeviceSynchronize();
  g_plans.clear();
}
