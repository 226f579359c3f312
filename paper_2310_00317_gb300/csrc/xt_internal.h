// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "xtgb.h"

struct xt_tracker;

namespace xt {

// ---------------------------------------------------------------------------
// Device lattice: a byte stream of 16-byte aligned records, one per non-marker
// element, in lattice order.  Record = 16-byte header + FP64 parameters padded
// to a multiple of 16 bytes.  Chunks are contiguous record ranges copied into
// shared memory by one bulk copy each.
struct RecHdr {
  uint16_t type;
  uint16_t order;
  uint16_t flags;   // REC_CURV: hxl != 0; REC_RAD: L_rad > 0
  uint16_t size16;  // record size in 16-byte units
  uint32_t elem;    // index of the element in the user's table
  uint32_t pad;
};
static_assert(sizeof(RecHdr) == 16, "record header is 16 bytes");
enum : uint16_t { REC_CURV = 1, REC_RAD = 2, REC_PURE = 4, REC_BEND = 8 };
// thick quadrupole: x is the focusing plane (k1 >= 0)
enum : uint16_t { REC_QF = 1 };
// thick bend: the full (exact) model; the full model with a gradient (kicks)
enum : uint16_t { REC_BFULL = 1, REC_BKICK = 2 };
// dipole edge: the non-linear model
enum : uint16_t { REC_ENL = 1, REC_EWEDGE = 2 };
// REC_PURE: knl0 == ksl0 == 0 and hxl == 0.  REC_BEND: hxl != 0, hxl == knl0,
// ksl0 == 0.  Without radiation these multipoles add the last Horner step
// straight into px, py (and a bend's -knl0 + hxl (1+delta) becomes hxl delta).

// Multipole record parameters (doubles after the header):
//   [0] hxl  [1] k0h = knl0 hxl / L_rad  [2] crl = crad L_rad  [3] ilr2 = 1/L_rad^2
//   [4] kql = kq L_rad  [5] L_rad  [6 + 2n] c_n = knl_n/n!  [7 + 2n] s_n = ksl_n/n!
// Drift: [0] L.  Cavity: [0] krf [1] lag [rad] [2] qv = q0 V/p0c.
// Edge: [0] r21 [1] r43.  Linear map: [0..35] M in (x,px,y,py,zeta,ptau),
// [36..41] d.  Aperture: [0] r^2 [1] half side of a square inside the circle
// (r (1 - 2^-20) / sqrt 2): |x|, |y| below it means inside, tested on the
// integer pipe.
enum { MP_HXL = 0, MP_K0H = 1, MP_CRL = 2, MP_ILR2 = 3, MP_KQL = 4, MP_LRAD = 5, MP_COEF = 6 };

struct Chunk {
  uint32_t off;    // byte offset in the record stream
  uint32_t bytes;  // multiple of 16
  uint32_t nrec;
  uint32_t pad;
};

// Reference-derived constants used by the kernels.
struct RefDev {
  double beta0, gamma0, bg0, ib0, twoib0, p0c, uc15, ig02, ip0c;  // ig02 = 1/gamma0^2, ip0c = 1/p0c
};

// Coefficients of the sine used by the RF cavity (Taylor series on |r| <= pi/4).
struct SinTab {
  double s[10];
  double c[11];
};

struct Lattice {
  std::vector<uint8_t> bytes;     // record stream
  std::vector<uint32_t> rec_off;  // byte offset of every record
  std::vector<uint32_t> rec_bytes;
  std::vector<int32_t> row_rec;   // per table row: its record's byte offset, -1 if it has none
  bool thick = false;             // a beam-beam, thick-quadrupole, bend or non-linear-edge record
  int64_t n_el = 0;               // rows in the user's table
  uint64_t hash = 0;
  std::vector<int64_t> flops;     // algorithmic FP64 flops of one traversal, per table row
};

struct Refc {
  double m0, q0, p0c, E0, beta0, gamma0, bg0, ib0, twoib0, crad, kq, uc15, ig02;
};

// e^(-j/64), j = 0..XT_EXPNEG_N - 1, stored after the photon spectrum's knots
// (the quantum model's e^(-nbar) for nbar < 16).
constexpr int XT_EXPNEG_N = 1025;

// Photons a warp samples together in shared memory per radiating slice
// (quantum radiation); more fall back to sampling by each particle.
constexpr int XT_PHOTON_CAP = 128;

// Host-side compilation (xt_lattice.cpp).
Refc ref_constants(const xt_reference& r);
int compile_lattice(const xt_element* table, int64_t n, const Refc& rc, Lattice* out, std::string* err);
void build_chunks(const Lattice& lat, uint32_t chunk_bytes, std::vector<Chunk>* out);
SinTab sin_table();
// Photon spectrum inverse-CDF table: knots (xi_i, F_i), i = 0..K-1.
void photon_table(std::vector<double>* xi, std::vector<double>* F, std::vector<int32_t>* guide);
constexpr int XT_SPEC_GUIDE = 4096;  // guide-table entries (uniform cells in the CDF)
int64_t flops_of_row(const xt_element& e, int rad_mode);

// ---------------------------------------------------------------------------
// Kernel parameter block (passed by value).
struct TrackArgs {
  const uint8_t* lat;
  const Chunk* chunks;
  int32_t n_chunks;
  int32_t n_el;
  int32_t chunk_bytes;  // buffer size per stage
  int32_t turn0;
  int32_t n_turns;
  int32_t pad0;
  double *x, *px, *y, *py, *zeta, *delta, *ptau, *rpp, *rvv;
  int32_t *state, *at_turn, *at_element;
  const int64_t* pid;
  const int32_t* idx;      // alive index list (compacted)
  const int32_t* n_alive;  // device scalar
  int32_t* tile_counter;   // device scalar, zeroed by the compaction
  int32_t* status;         // device scalar: 0 ok, else XT_ERR_* code
  const volatile int32_t* cancel;  // host-mapped flag
  int64_t max_cycles;
  uint64_t seed;
  const double* spec_xi;
  const double* spec_F;
  const int32_t* spec_guide;
  int32_t spec_k;
  int32_t pad1;
  RefDev ref;
  SinTab sn;
};

// One pass of the table for a few particles with their state recorded after
// every table row (one thread per particle; records read from global memory).
struct MonitorArgs {
  const uint8_t* lat;
  const int32_t* row_off;  // per table row: record offset in lat, -1 if none
  int32_t n_el;
  int32_t turn;
  int64_t n;
  double *x, *px, *y, *py, *zeta, *delta, *ptau, *rpp, *rvv;
  int32_t *state, *at_turn, *at_element;
  const int64_t* pid;
  double* out;  // [row][8][n]: x, px, y, py, zeta, ptau, delta, state
  uint64_t seed;
  const double* spec_xi;
  const double* spec_F;
  const int32_t* spec_guide;
  int32_t spec_k;
  int32_t pad0;
  RefDev ref;
  SinTab sn;
};
int launch_monitor(const MonitorArgs& a, int rad, void* stream);

// Loss-location refinement (one thread per particle).  Tables built on the
// host per tracker: for every table row its record offset in `lat` (-1 for a
// marker), its entrance position and reference frame (cos, sin, dx, dy:
// lab = R(-th) local + d), the previous aperture row and the index of its
// laboratory-frame polygon (-1 if none or unusable).
struct RefineArgs {
  const uint8_t* lat;
  const int32_t* row_off;
  const double* spos;      // n_el + 1 entries (the last is the table length)
  const double* frame;     // 4 per row
  const int32_t* prev_ap;
  const int32_t* poly_idx;
  const double* polys;     // n_angles x (x, y) per polygon
  int32_t n_el;
  int32_t n_angles;
  double ds;
  const double *x, *px, *y, *py, *zeta, *delta, *ptau, *rpp, *rvv;
  const int32_t *state, *at_element;
  double* s_loss;
  int64_t n;
  RefDev ref;
  SinTab sn;
};

int launch_refine(const RefineArgs& a, void* stream);

// Constant table of the special functions (beam-beam kick, thick elements;
// XT_SPECIAL_N doubles, see special_table) for the current device's
// constant memory.
#define XT_SPECIAL_N 278
#define XT_SPECIAL_FACT 41    // 1/n!, n = 0..21
#define XT_SPECIAL_ASIN 63    // asin(v)/v series coefficients, n = 0..13
#define XT_SPECIAL_RECIP 77   // 1/k, k = 0..200 (entry 0 unused): the photon-count recurrence
void special_table(double* out);
int upload_special_table(const double* tab);

// Batched-seed variant: per-seed lattice and particle pointers in device arrays.
struct SeedDev {
  const uint8_t* lat;
  const Chunk* chunks;
  int32_t n_chunks;
  int32_t n_el;
  double *x, *px, *y, *py, *zeta, *delta, *ptau, *rpp, *rvv;
  int32_t *state, *at_turn, *at_element;
  const int64_t* pid;
  int64_t n;
};

struct BatchArgs {
  const SeedDev* seeds;
  const int32_t* seed_order;   // seeds sorted by particle count, descending
  const int64_t* tile_prefix;  // prefix sum of tiles in seed_order (n_seeds+1)
  const int32_t* idx;          // per-seed compacted alive lists, concatenated
  const int64_t* idx_base;     // start of each seed's list in idx
  const int32_t* n_alive;      // per seed
  int32_t* tile_counter;
  int32_t* status;
  const volatile int32_t* cancel;
  const int32_t* turn_base;    // device scalar: first turn of the call
  int32_t turn_off;            // this segment's offset from turn_base
  int32_t n_seeds;
  int32_t chunk_bytes;
  int32_t n_turns;
  int64_t max_cycles;
  uint64_t seed;
  const double* spec_xi;
  const double* spec_F;
  const int32_t* spec_guide;
  int32_t spec_k;
  int32_t pad1;
  RefDev ref;
  SinTab sn;
};

// Launchers (xt_track.cu).  Return a cudaError_t as int.
int launch_compact(const int32_t* state, int64_t n, int32_t* block_counts, int32_t* idx,
                   int32_t* n_alive, int32_t* tile_counter, void* stream);
// kind = radiation mode (XT_RAD_*) + 3 when the table has thick rows
// (Lattice::thick): it picks the kernel instantiation.
int launch_track(const TrackArgs& a, int kind, int block, int grid, size_t smem, void* stream);
int track_occupancy(int kind, int block, size_t smem, int* blocks_per_sm);
int launch_compact_batched(const SeedDev* seeds_dev, int32_t n_seeds, const int64_t* idx_base_dev,
                           int32_t* idx, int32_t* n_alive, int32_t* counts, int64_t max_n, void* stream);
int launch_tile_prefix(const int32_t* n_alive, const int32_t* order, int32_t n_seeds,
                       int64_t* tile_prefix, int32_t* tile_counter, void* stream);
int launch_set_int(int32_t* dst, int32_t value, void* stream);
int launch_track_batched(const BatchArgs& a, int kind, int block, int grid, size_t smem,
                         void* stream);
int batched_occupancy(int kind, int block, size_t smem, int* blocks_per_sm);
int device_sm_count(int* n);
int device_smem_optin(int* bytes);
int launch_fp64_probe(double* out, int grid, int block, int iters, int variant, int* chains, void* stream);

size_t track_smem_bytes(int block, int chunk_bytes, int kind);

// Launch parameters of a tracker for the allocation-free entry point
// (xt_api.cpp): fills everything but the scratch pointers, allocates nothing.
int noalloc_prepare(xt_tracker* t, const xt_particles* p, int64_t n_turns, TrackArgs* a, int* block,
                    int* grid, size_t* smem, int* seg, int* rad);
void set_error(const std::string& msg);

}  // namespace xt
