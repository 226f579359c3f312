/*
 * xtgb.h -- C ABI of the GB300-native FP64 symplectic tracker.
 *
 * Element-by-element single-particle tracking of a particle ensemble through a
 * circular-accelerator lattice for many turns, the data-parallel hot path of the
 * Xsuite paper (Iadarola et al., "Xsuite: an integrated beam physics simulation
 * framework"):
 *   - a beam line is a sequence of element objects tracked turn after turn with
 *     thin-lens integration, compiled into one kernel that tracks the whole line
 *     on the GPU (section "Lattice modelling and single particle tracking");
 *   - aperture elements stop the tracking of particles found outside and record
 *     where they were lost (section "Particle-matter interaction and collimation
 *     studies");
 *   - synchrotron radiation in a "mean" and a "quantum" model for thin elements
 *     (section "Synchrotron radiation models and compensation").
 *
 * The paper prints no formulas.  The maps are the thin-lens Hamiltonian maps
 * with MAD-X sign conventions; their exact operation order is fixed (see the
 * element list below) so that results are reproducible bit for bit.
 *
 * Conventions for every function:
 *   - returns XT_OK (0) or a negative XT_ERR_* code; xt_last_error() gives a
 *     message for the calling thread.  No C++ exception crosses this ABI.
 *   - "device pointer" = memory of the current CUDA device (cudaMalloc or a
 *     PyTorch CUDA tensor); "host pointer" = ordinary or pinned host memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *     take a stream are asynchronous: the caller synchronises before reading.
 *   - All floating-point arithmetic of the tracking path is IEEE FP64.
 */
#ifndef XTGB_H
#define XTGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* Status codes                                                              */
#define XT_OK 0
#define XT_ERR_INVALID -1      /* bad argument (null pointer, size, range)    */
#define XT_ERR_UNSUPPORTED -2  /* unknown element type or multipole order > 10 */
#define XT_ERR_CUDA -3         /* a CUDA runtime call failed                   */
#define XT_ERR_TIMEOUT -4      /* the per-launch cycle budget ran out           */
#define XT_ERR_CANCELLED -5    /* xt_cancel() was called during tracking         */
#define XT_ERR_NOMEM -6        /* device or host allocation failed              */

/* ------------------------------------------------------------------------ */
/* Lattice table                                                             */
/* Element types (row.type).  Parameters row.p[...]:                         */
#define XT_MARKER 0     /* no parameters; no effect                           */
#define XT_DRIFT 1      /* p[0] = length L [m].  Exact drift:
                           pz = sqrt((1+delta)^2 - px^2 - py^2),
                           x += px L/pz, y += py L/pz,
                           zeta += L - (1+delta)/rvv * L/pz;
                           (1+delta)^2 - px^2 - py^2 outside (0, inf) -> lost
                           with state -2, coordinates unchanged.               */
#define XT_MULTIPOLE 2  /* row.order = N (0..10); p[0..10] = knl_n [m^-n],
                           p[11..21] = ksl_n, p[22] = hxl [rad],
                           p[23] = L_rad [m] (>= 0).  Thin kick:
                           b = sum_n (knl_n + i ksl_n)(x + i y)^n / n!,
                           px -= Re b, py += Im b; if hxl != 0:
                           px += hxl (1+delta) - knl0 hxl x / L_rad,
                           zeta -= hxl x / rvv.  Radiation acts after the kick
                           when enabled and L_rad > 0.                         */
#define XT_CAVITY 3     /* p[0] = voltage V [V], p[1] = frequency f [Hz],
                           p[2] = lag [deg].  ptau += q0 V sin(lag - 2 pi f
                           zeta/(beta0 c)) / p0c, then delta, rpp, rvv.        */
#define XT_DIPEDGE 4    /* p[0] = h [1/m], p[1] = e1 [rad], p[2] = hgap [m],
                           p[3] = fint, p[4] = model (0 linear, 1 non-linear,
                           2 exact wedge), p[5] = face (0 entrance, 1 exit;
                           models 1 and 2).
                           Linear edge: px += h tan(e1) x,
                           py -= h tan(e1 - psi) y,
                           psi = 2 h hgap fint (1 + sin^2 e1) / cos e1.
                           Non-linear edge (section "Lattice modelling and
                           single particle tracking"): the canonical map of
                           the generating function with the fringe term
                           (h/2) y^2 tan(e1 + s atan(px/pz)), s = +1 at the
                           entrance and -1 at the exit (py solved by
                           fixed-point iteration to convergence; x, y, zeta
                           shifted), the wedge kick px += h tan(e1) x, and
                           the finite-extent correction
                           py += h (tan e1 - tan(e1 - psi)) y; its
                           linearisation is the linear edge.
                           Exact wedge: the same fringe taken on the face
                           itself (face angle 0 in the face's frame) between
                           two exact changes of plane: at the entrance a
                           straight line from the plane normal to the orbit
                           to the face, then the circle in the field h back
                           to the normal plane; at the exit the mirror
                           sequence.  Its linearisation is the linear edge.
                           Models 1 and 2: lost with state -2 if pz is not
                           real or a plane is not reached; no inverse is
                           formed for them in loss refinement.             */
#define XT_LINEARMAP 5  /* p[0..35] = M (row-major 6x6), p[36..41] = d, acting
                           on (x, px, y, py, zeta, pzeta), pzeta = ptau/beta0:
                           v -> M v + d, then delta, rpp, rvv from ptau.      */
#define XT_APERTURE 6   /* p[0] = radius r [m].  Circular aperture: lost with
                           state 0 if x^2 + y^2 > r^2, state -1 if x or y is not
                           finite.  A point on the circle survives.           */
/* Misalignments and tilts are changes of the reference system (section
   "Lattice modelling and single particle tracking" of the paper): a shifted or
   tilted element is wrapped in a shift/rotation and its inverse.            */
#define XT_XYSHIFT 7    /* p[0] = dx, p[1] = dy [m].  x -= dx, y -= dy.        */
#define XT_SROTATION 8  /* p[0] = angle theta [rad] about the reference orbit:
                           x' = x cos + y sin, y' = -x sin + y cos, and the same
                           for (px, py); cos and sin of theta are taken once on
                           the host.                                           */
#define XT_APERTURE_RECT 9     /* p[0] = x_min, p[1] = x_max, p[2] = y_min,
                           p[3] = y_max [m] (x_min <= x_max, y_min <= y_max):
                           lost with state 0 unless x_min <= x <= x_max and
                           y_min <= y <= y_max, state -1 if x or y is not
                           finite.  The boundary survives.                     */
#define XT_APERTURE_ELLIPSE 10 /* p[0] = a, p[1] = b [m] (> 0): lost with state 0
                           if x^2 (1/a^2) + y^2 (1/b^2) > 1 (1/a^2, 1/b^2 taken
                           once on the host), state -1 if x or y is not
                           finite.                                             */
#define XT_BEAMBEAM4D 11 /* 4D weak-strong beam-beam lens (section "Beam-beam
                           interactions"): p[0] = q_s N_s, the charge [e] times
                           the number of particles of the strong bunch, p[1] =
                           its speed beta_s (0 < beta_s <= 1, moving against
                           the tracked beam), p[2], p[3] = sigma_x, sigma_y
                           [m] (> 0), p[4], p[5] = its centre x_c, y_c [m].
                           px += K f_x, py += K f_y with
                           K = 2 q0 q_s N_s (r_e m_e c^2 / p0 c)
                               (1 + beta0 beta_s) / (beta0 + beta_s)
                           and f the field shape of a unit bi-Gaussian line
                           charge at (x - x_c, y - y_c): Bassetti-Erskine with
                           the Faddeeva function (round-beam closed form when
                           sigma_x^2, sigma_y^2 agree to 1e-10; the linear
                           field within (dx/sigma_x)^2 + (dy/sigma_y)^2 < 1e-10
                           of the centre).  Independent of zeta and delta.   */
#define XT_QUAD 12       /* p[0] = k1 [m^-2] (> 0 focuses in x), p[1] = length
                           L [m] (finite, >= 0; L = 0 has no effect).  Thick
                           quadrupole (section "Lattice modelling and single
                           particle tracking"): the exact flow of
                           (px^2 + py^2) / (2 (1+delta)) + k1 (x^2 - y^2) / 2,
                           harmonic with w^2 = |k1| / (1+delta) (cos/sin in
                           the focusing plane, cosh/sinh in the other); zeta
                           gains L (1 - 1/rvv) minus the integral of
                           (px^2 + py^2) / (2 rvv (1+delta)^2) over the body,
                           in closed form.  Delta and ptau are unchanged.
                           Loss refinement steps through it like a drift.    */
#define XT_BEND 13       /* Thick sector bend (section "Lattice modelling and
                           single particle tracking": a full map for small
                           machines, an expanded one for large machines and
                           small bending angles).  p[0] = k0 = B / (B rho)
                           [1/m], p[1] = frame curvature h [1/m] (k0 = h on
                           the design orbit; h = 0 is a straight frame),
                           p[2] = reference length L [m] (finite, >= 0),
                           p[3] = gradient k1 [m^-2], p[4] = model: 0
                           expanded, 1 full, p[5] = gradient kicks n of the
                           full model (integer 0..64, 0 means 1).
                           Expanded: the exact flow of
                           (px^2 + py^2) / (2 (1+delta)) - h x (1+delta)
                           + k0 (x + h x^2 / 2) + k1 (x^2 - y^2) / 2, with
                           zeta' = 1 - (1/rvv)(1 + h x + (px^2 + py^2) /
                           (2 (1+delta)^2)).  Full: the exact motion in the
                           uniform field through the sector (arc of a circle
                           in the horizontal plane, straight in y); lost with
                           state -2 if the particle cannot reach the exit
                           plane.  A gradient in the full model has no
                           closed form: the body is cut into n slices, each
                           an exact half body, a thin kick px -= k1 (L/n) x,
                           py += k1 (L/n) y and an exact half body (second
                           order in L/n; -L inverts it).  Delta and ptau are
                           unchanged.  Loss refinement steps through it like
                           a drift, except a full bend with a gradient, which
                           it passes whole (its slices are not a flow).     */
#define XT_SPACECHARGE 14 /* Frozen space-charge lens (section "Space charge",
                           frozen model): p[0] = peak line density lambda0
                           [particles/m], p[1] = sigma_z [m] (> 0 a Gaussian
                           bunch; 0 a coasting beam), p[2], p[3] = sigma_x,
                           sigma_y [m] (> 0), p[4] = length L [m] of ring the
                           lumped lens stands for, p[5], p[6] = beam centre.
                           px += K g f_x, py += K g f_y with
                           K = 2 r_c lambda0 L / (beta0^2 gamma0^3),
                           r_c = q0^2 r_e m_e / m0, g = exp(-zeta^2 /
                           (2 sigma_z^2)) (1 when coasting) and f the field
                           shape of XT_BEAMBEAM4D at (x - x_c, y - y_c).
                           Independent of delta.                            */

#define XT_MAX_ORDER 10
#define XT_NPARAM 48

/* One row of the flat lattice table (392 bytes, 8-byte aligned).            */
typedef struct {
  int32_t type;
  int32_t order;
  double p[XT_NPARAM];
} xt_element;

/* Reference particle: rest energy [eV], charge [e], reference momentum
   p0c [eV].  Derived: E0 = sqrt(p0c^2 + mass0^2), beta0 = p0c/E0.            */
typedef struct {
  double mass0;
  double q0;
  double p0c;
} xt_reference;

/* ------------------------------------------------------------------------ */
/* Particles: structure of arrays, n entries each, all DEVICE pointers,
   borrowed by the call (the caller owns them).
   x [m], px = Px/P0, y [m], py, zeta = s - beta0 c t [m],
   delta = (P-P0)/P0, ptau = (E-E0)/(P0 c), rpp = 1/(1+delta), rvv = beta/beta0
   (delta, ptau, rpp, rvv must be consistent; they are updated together).
   state: 1 alive; 0 lost at an aperture; -1 lost with a non-finite x or y;
   -2 lost in a drift (no longitudinal momentum); -3 lost at the end-of-turn
   guard (|x| or |y| > 1 m).  Lost particles keep the coordinates they had at
   the loss; at_turn (absolute, 0-based) and at_element record where.
   Survivors end with at_turn = start_turn + n_turns, at_element = 0.
   particle_id keys the quantum-radiation random numbers.                    */
typedef struct {
  double *x, *px, *y, *py, *zeta, *delta, *ptau, *rpp, *rvv;
  int32_t *state, *at_turn, *at_element;
  const int64_t *particle_id;
  int64_t n;
} xt_particles;

/* ------------------------------------------------------------------------ */
/* Options                                                                   */
#define XT_RAD_OFF 0
#define XT_RAD_MEAN 1     /* deterministic energy loss per radiating element   */
#define XT_RAD_QUANTUM 2  /* Poisson photon emission, Philox4x64-10 keyed by
                             (seed; particle_id, turn, element, draw)          */
typedef struct {
  int32_t radiation;      /* XT_RAD_*                                          */
  int32_t block;          /* threads per block: 0 = default, else 32..256, %32 */
  int32_t chunk_bytes;    /* lattice staging chunk: 0 = default, else 1 KiB ..
                             48 KiB, multiple of 16                             */
  int32_t segment_turns;  /* turns per launch between compactions of the alive
                             set: 0 = default                                   */
  uint64_t seed;          /* quantum-radiation key                              */
  int64_t max_cycles;     /* per-launch clock64 budget per warp: 0 = none; when
                             exceeded tracking stops at a turn boundary and
                             xt_sync_status() returns XT_ERR_TIMEOUT            */
} xt_options;

/* Fills `opt` with the defaults.                                            */
void xt_options_default(xt_options* opt);

/* ------------------------------------------------------------------------ */
/* Tracker                                                                   */
typedef struct xt_tracker xt_tracker;

/* Compiles the host table (n_elements rows, host pointer, copied; the caller
   may free it afterwards) into the device lattice of the current device.
   Errors: XT_ERR_INVALID (null pointer, n_elements < 1 or > 2^24, reference
   with mass0 <= 0 or p0c <= 0, options out of range), XT_ERR_UNSUPPORTED
   (unknown type, multipole order outside 0..10), XT_ERR_CUDA/NOMEM.          */
int xt_tracker_create(const xt_element* table, int64_t n_elements, const xt_reference* ref,
                      const xt_options* opt, xt_tracker** out);

/* Frees the tracker and its device memory (synchronises the device).        */
void xt_tracker_destroy(xt_tracker* tr);

/* Replaces the tracker's launch options (radiation mode, block, chunk,
   segment, seed, budget).  Same range checks as create.                      */
int xt_tracker_set_options(xt_tracker* tr, const xt_options* opt);
int xt_tracker_get_options(const xt_tracker* tr, xt_options* opt);

/* Tracks particles p (device pointers, updated in place) for n_turns turns
   starting at absolute turn start_turn (>= 0, start_turn + n_turns < 2^31).
   Asynchronous on `stream`.  Particles with state != 1 are not touched.
   Tracking runs as launches of `segment_turns` turns; between launches the
   alive particles are compacted into an index list so lost particles cost
   nothing afterwards.  Results do not depend on the segmentation, block or
   chunk size: track(a) followed by track(b) from turn a equals track(a+b)
   bit for bit.  Uses the tracker's own workspace (grown on demand with
   cudaMalloc, so the first call with a larger n must not be inside a stream
   capture); calls on one tracker must be ordered on one stream.
   Errors: XT_ERR_INVALID, XT_ERR_CUDA, XT_ERR_NOMEM.                        */
int xt_track(xt_tracker* tr, const xt_particles* p, int64_t start_turn, int64_t n_turns,
             void* stream);

/* Same as xt_track with HOST particle arrays (pointer fields of `p` are host
   pointers): copies them to the tracker's device buffers, tracks, copies the
   results back and synchronises `stream` before returning.                  */
int xt_track_host(xt_tracker* tr, const xt_particles* p, int64_t start_turn, int64_t n_turns,
                  void* stream);

/* Same tracking as xt_track, for callers that cannot allocate device memory
   while they track (an application whose device memory is owned by its own
   allocator or budget, or a real-time loop that cannot wait for cudaMalloc).
   There is no counterpart in the paper.  xt_track grows a per-tracker
   workspace with cudaMalloc; this call allocates nothing: its scratch (alive
   list, counts, counters) is a fixed static device array of
   XT_NOALLOC_MAX_PARTICLES entries (about 4 MiB, held by every GPU that loads
   the library until exit).  The caller passes the tracker (created
   beforehand) and the particles.  n > XT_NOALLOC_MAX_PARTICLES ->
   XT_ERR_INVALID.  The first call on a device looks up the array's device
   address (once per device, with that device current); make that first call
   before any stream capture.  All calls share the one array: calls that
   overlap on the GPU (other streams, other trackers) race.  The current
   device must be the tracker's (else XT_ERR_INVALID).  Cycle budget and
   cancel act as in xt_track; their status goes to the array's status word,
   which xt_noalloc_status() reads.                                         */
#define XT_NOALLOC_MAX_PARTICLES 1048576
int xt_track_noalloc(xt_tracker* tr, const xt_particles* p, int64_t start_turn, int64_t n_turns,
                     void* stream);

/* Outcome of the last xt_track_noalloc call on the current device: XT_OK,
   XT_ERR_TIMEOUT (cycle budget spent) or XT_ERR_CANCELLED.  Synchronises
   `stream`, reads the static array's status word and clears it; allocates
   nothing.  No counterpart in the paper.                                   */
int xt_noalloc_status(void* stream);

/* Synchronises `stream` and returns the status of the tracker's launches
   since the last call: XT_OK, XT_ERR_TIMEOUT or XT_ERR_CANCELLED; clears it. */
int xt_sync_status(xt_tracker* tr, void* stream);

/* Asks running and future launches of this tracker to stop at the next turn
   boundary (host-visible flag; thread-safe).  xt_reset_cancel() clears it.   */
int xt_cancel(xt_tracker* tr);
int xt_reset_cancel(xt_tracker* tr);

/* Monitor: one pass of the table (turn number `turn`, which keys the quantum
   radiation's random numbers) for the particles in device buffers, with their
   state written after every table row: out (device, n_elements * 8 * n
   doubles, caller-owned) receives for row i, coordinate c of (x, px, y, py,
   zeta, ptau, delta, state) and particle j the value out[(i * 8 + c) * n + j]
   (the state as a double: 1 alive, else the loss code).  The particles are
   advanced exactly as one turn of xt_track would advance them (bit for bit),
   under the tracker's radiation mode.  It serves the lattice functions along
   the line and the energy-loss compensation of section "Twiss module"; at
   most XT_MONITOR_MAX_PARTICLES particles (else XT_ERR_INVALID).  Async on
   `stream`.                                                                */
#define XT_MONITOR_MAX_PARTICLES 4096
int xt_track_monitor(xt_tracker* tr, const xt_particles* particles, int64_t turn, double* out, void* stream);

/* Algorithmic FP64 flops of one traversal of every table row, for roofline
   accounting (FMA = 2, add or multiply = 1, square root, divide and sine = 1,
   compares 0), under the tracker's radiation mode: flops_per_element[i] for
   row i, n_elements = the table's length (else XT_ERR_INVALID).  Host only. */
int xt_element_flops(const xt_tracker* tr, int64_t* flops_per_element, int64_t n_elements);

/* Event timing of the tracking kernel launches on their stream: after
   xt_set_profiling(tr, 1) every tracking launch of this tracker is bracketed
   by CUDA events; xt_kernel_time() synchronises them and returns the summed
   duration [ms] and the number of launches since the last query, then
   restarts the count.  Profiling off (default) records nothing.            */
int xt_set_profiling(xt_tracker* tr, int enable);
int xt_kernel_time(xt_tracker* tr, double* total_ms, int64_t* launches);

/* Diagnostic: FP64 fma throughput of the current device [flop/s]: the
   fastest of twelve probe launches (8 or 16 independent fma chains per
   thread, shared or per-chain operands, 4, 8 or 16 blocks of 128 threads
   per SM) on `stream`, blocking until done; *elapsed_ms is that launch's
   duration.  Allocates a scratch buffer with cudaMalloc.                   */
int xt_fp64_peak(double* flops_per_s, double* elapsed_ms, void* stream);

/* Picks block size, chunk size and segment length by timing short probe runs
   on a copy of `probe` (device particles, not modified) for `probe_turns`
   turns, and stores them in the tracker's options.  Results are cached per
   (lattice hash, particle count, radiation mode) in the process.           */
int xt_autotune(xt_tracker* tr, const xt_particles* probe, int64_t probe_turns, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched error seeds: n_seeds trackers (one lattice each, same reference and
   radiation mode) with their own particle sets, tracked in ONE persistent
   launch per segment: CTAs pull (seed, 32-particle tile) work items from a
   queue ordered largest-seed first.  Launch parameters come from trackers[0].
   When `graph` != 0 the whole multi-segment sequence is captured once into a
   CUDA graph (cached per argument set) and replayed.  Same result semantics
   as calling xt_track on each seed.                                         */
int xt_track_batched(xt_tracker* const* trackers, const xt_particles* particles, int32_t n_seeds,
                     int64_t start_turn, int64_t n_turns, int32_t graph, void* stream);

/* Synchronises `stream` and returns the status word of the batched launches
   made with exactly these arguments (XT_OK, XT_ERR_TIMEOUT, XT_ERR_CANCELLED),
   then clears it.  XT_ERR_INVALID if no such batched launch was made.       */
int xt_batched_sync_status(xt_tracker* const* trackers, const xt_particles* particles, int32_t n_seeds,
                           void* stream);

/* Frees the device memory and graphs cached by xt_track_batched (synchronises
   the device).  Call before destroying trackers used in batched launches.    */
void xt_batched_release(void);

/* ------------------------------------------------------------------------ */
/* Loss-location refinement (section "Particle-matter interaction and
   collimation studies" of the paper: backtracking and a polygonal
   interpolation of the aperture).
   For every particle with state 0 lost at an aperture row e (XT_APERTURE,
   XT_APERTURE_RECT, XT_APERTURE_ELLIPSE), s_loss[i] receives the position
   [m from the start of the table, the loss turn not included] where its
   trajectory first leaves the aperture between the previous aperture row q
   and e, to within ds [m]:
   - the aperture between q and e is the polygon interpolated linearly in s
     between the two apertures' polygons; each polygon joins the boundary
     points met by n_angles rays at angles 2 pi k / n_angles from the
     aperture's own frame origin (which must lie inside it), taken to the
     laboratory frame through the shift and rotation rows before the row;
   - the particle is backtracked from its loss coordinates to the exit of q
     with the inverse maps (drift of -L, kicks and frame changes undone),
     then tracked forward again with every drift cut into steps of at most
     ds; s_loss is the first step end found outside the interpolated
     polygon, or the position of e if none is;
   - radiation is not reversed (the maps between two apertures are taken
     without it), and a linear-map row between q and e makes the particle's
     result NaN.
   Other particles get NaN.  Particles are DEVICE arrays as for xt_track and
   are not modified; s_loss is a DEVICE array of n doubles.  Errors:
   XT_ERR_INVALID (null pointer, ds <= 0, n_angles outside 8..1024, no
   aperture row in the table).  The tables are built on the first call (and
   when n_angles changes) and kept by the tracker; the call is asynchronous
   on `stream` afterwards.                                                   */
int xt_refine_losses(xt_tracker* tr, const xt_particles* particles, double ds, int32_t n_angles,
                     double* s_loss, void* stream);

/* ------------------------------------------------------------------------ */
/* Dynamic-aperture surrogate network.  The paper lists dynamic-aperture
   estimates based on machine learning among Xsuite's applications (section
   "Lattice modelling and single particle tracking"); the network is this
   project's: MLP 16 -> 256 -> 256 -> 256 -> 256 -> 2 with GELU (erf by
   Hastings' rational approximation, Abramowitz & Stegun 7.1.26, within
   1.5e-7), inputs = 6 normalised initial coordinates + 10 lattice-error
   descriptors,
   outputs = (survival logit, normalised log loss turn).  bfloat16 weights,
   inputs, activations and back-propagated dZ; FP32 accumulation on the
   tensor cores, FP32 bias/GELU/head/loss; FP32 master weights with Adam
   (beta1 0.9, beta2 0.999, eps 1e-8).
   Flat parameter layout (XS_N_PARAMS floats): W1 (256x16, row = output unit),
   b1 (256), W2 (256x256), b2, W3, b3, W4, b4, W5 (2x256), b5 (2).
   Errors are reported by xs_last_error().                                   */
#define XS_N_PARAMS 202242
typedef struct xs_mlp xs_mlp;

/* Allocates the network on the current device, weights uniform in
   +-1/sqrt(fan_in) from `seed`.                                             */
int xs_mlp_create(uint64_t seed, xs_mlp** out);
void xs_mlp_destroy(xs_mlp* net);
/* Copies XS_N_PARAMS FP32 parameters from / to HOST memory (synchronous);
   set_params also resets the Adam moments and step count.                  */
int xs_mlp_set_params(xs_mlp* net, const float* params, int64_t n, void* stream);
int xs_mlp_get_params(xs_mlp* net, float* params, int64_t n, void* stream);
/* Inference: X (DEVICE, B x 16 FP32, row-major) -> out (DEVICE, B x 2).      */
int xs_mlp_forward(xs_mlp* net, const float* X, float* out, int64_t B, void* stream);
/* Forward + backward without an update.  y (survived 1/0), t (normalised log
   loss turn), mask (1 where t is defined) are DEVICE FP32 arrays of B.
   loss = mean BCE(logit, y) + lam * sum mask (pred - t)^2 / max(sum mask, 1).
   grad_out (DEVICE, XS_N_PARAMS) and loss_out (DEVICE scalar) may be NULL.  */
int xs_mlp_loss_grad(xs_mlp* net, const float* X, const float* y, const float* t, const float* mask,
                     int64_t B, float lam, float* grad_out, float* loss_out, void* stream);
/* One Adam step on the batch; loss_out (DEVICE scalar) may be NULL.         */
int xs_mlp_train_step(xs_mlp* net, const float* X, const float* y, const float* t, const float* mask,
                      int64_t B, float lr, float lam, float* loss_out, void* stream);
const char* xs_last_error(void);

/* Surrogate-guided dynamic-aperture scan glue.  Grid points are ray-major
   (i = ray * n_r + k, radius index k increasing outward); the DA of a ray is
   the number of radii before its first lost point.  out2 is the network
   output (DEVICE, n_rays*n_r x 2), state the particles' state array (DEVICE).
   xs_da_select, first pass (widen == NULL): per ray r_lo = first point whose
   survival probability is below 1 - p_lo (written to r_lo[ray], n_r if none);
   points k in [r_lo - margin, r_lo + window] get state 1 (to be tracked by
   xt_track), all others XS_STATE_PREDICTED.  Later passes (widen != NULL,
   da_prev = the previous pass's da): state 1 -> XS_STATE_SURVIVED; on rays
   with widen[ray] == XS_WIDEN_INWARD the predicted points in
   [da_prev - margin, da_prev - 1], on rays with widen[ray] == XS_WIDEN_VERIFY
   those in [da_prev - margin, da_prev + margin], become 1 (window unused).
   xs_da_combine: da[ray] = first lost point (tracked: state <= 0; predicted:
   logit < 0; out2 may be NULL when every point was tracked, then predicted
   points count as survivors); widen[ray] (may be NULL) = XS_WIDEN_VERIFY if
   that point is predicted, XS_WIDEN_INWARD if it is tracked but its inner
   neighbour is predicted (the boundary may lie further in), else 0.
   Both return XT_ERR_INVALID for a null required pointer, negative sizes,
   margin or window, or p_lo outside (0, 0.5); all pointers stay owned by the
   caller and the calls only enqueue work on `stream`.                      */
#define XS_WIDEN_INWARD 1
#define XS_WIDEN_VERIFY 2
#define XS_STATE_PREDICTED 2
#define XS_STATE_SURVIVED 3
int xs_da_select(const float* out2, int32_t n_rays, int32_t n_r, float p_lo, int32_t margin, int32_t window,
                 const int32_t* widen, const int32_t* da_prev, int32_t* state, int32_t* r_lo, void* stream);
int xs_da_combine(const float* out2, const int32_t* state, int32_t n_rays, int32_t n_r, int32_t* da,
                  int32_t* widen, void* stream);
const char* xs_da_last_error(void);

/* ------------------------------------------------------------------------ */
/* Message of the last failed call on this thread ("" if none).              */
const char* xt_last_error(void);
/* Library version string.                                                   */
const char* xt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* XTGB_H */
