// Persistent FP64 tracking kernels for sm_103a.
//
// One thread per particle.  Each warp pulls 32-particle tiles from a work
// counter, loads the tile's state into registers, tracks it for all turns of
// the launch, and writes it back.  The lattice is a stream of 16-byte aligned
// records; each warp stages it chunk by chunk into its own pair of shared
// memory buffers with cp.async.bulk (completion on an mbarrier), so the
// element parameters are read as warp-uniform shared-memory broadcasts while
// the next chunk is in flight.  Lost particles are removed between launches by
// an order-preserving compaction, because on this GPU a masked lane costs the
// FP64 pipe as much as an active one.
//
// Every FP64 operation below follows the fixed operation order of the maps
// (explicit fma where the map says fma, nothing contracted: -fmad=false), so the
// results equal those of a plain IEEE implementation of the same maps bit for
// bit.  Comparisons that only decide a loss are done on the integer pipe with
// the IEEE bit patterns (monotone for non-negative doubles), keeping the
// scarce FP64 pipe for arithmetic.
#include <cuda_runtime.h>
#include <cstdint>

#include "xt_internal.h"

namespace xt {

#define FULL_MASK 0xffffffffu
#define XT_MAX_BLOCK 256
static const int64_t STAGE_WAIT_LIMIT = 4000000000LL;  // clock cycles (~2 s)
static const int64_t POLL_INTERVAL = 1000000LL;        // cycles between cancel polls

// ---------------------------------------------------------------------------
// Shared-memory staging primitives (inline PTX).
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Per-warp double buffer.  Lane 0 issues; all lanes wait.
struct Stage {
  uint8_t* buf[2];
  uint64_t* bar[2];
  uint32_t parity;   // bit b: parity of the next completion of buffer b
  uint32_t pending;  // bit b: a copy into buffer b is in flight
};

__device__ __forceinline__ void stage_issue(Stage& s, int b, const uint8_t* src, uint32_t bytes, int lane) {
  if (lane == 0) {
    fence_proxy_async();  // order earlier generic reads of the buffer before the async write
    uint64_t* bar = b ? s.bar[1] : s.bar[0];
    mbar_expect_tx(bar, bytes);
    bulk_copy_g2s(b ? s.buf[1] : s.buf[0], src, bytes, bar);
  }
  s.pending |= 1u << b;
}

// Bounded wait; returns false if the copy did not land within the limit.
__device__ __forceinline__ bool stage_wait(Stage& s, int b) {
  const uint32_t par = (s.parity >> b) & 1u;
  uint64_t* bar = b ? s.bar[1] : s.bar[0];
  bool ok = mbar_try_wait(bar, par);
  if (!ok) {
    const int64_t t0 = clock64();
    while (!(ok = mbar_try_wait(bar, par))) {
      if (clock64() - t0 > STAGE_WAIT_LIMIT) break;
    }
  }
  ok = __all_sync(FULL_MASK, ok);
  if (ok) {
    s.parity ^= 1u << b;
    s.pending &= ~(1u << b);
  }
  return ok;
}

__device__ __forceinline__ void stage_drain(Stage& s) {
  for (int b = 0; b < 2; b++)
    if (s.pending & (1u << b)) stage_wait(s, b);
}

// ---------------------------------------------------------------------------
// Integer-pipe classification of IEEE doubles.  The bit pattern of |v| is
// taken in inline PTX: written as a plain mask, the compiler recognises |v|
// (or a floating-point class test) and issues it on the FP64 pipe, where it
// costs a full slot.
__device__ __forceinline__ uint64_t dbits(double v) { return (uint64_t)__double_as_longlong(v); }
__device__ __forceinline__ uint64_t abs_bits(double v) {
  uint64_t r;
  asm("and.b64 %0, %1, 0x7FFFFFFFFFFFFFFF;" : "=l"(r) : "l"(dbits(v)));
  return r;
}
__device__ __forceinline__ bool is_finite(double v) { return abs_bits(v) < 0x7FF0000000000000ull; }
// |v| <= 1 (false for NaN)
__device__ __forceinline__ bool abs_le_one(double v) { return abs_bits(v) <= 0x3FF0000000000000ull; }
// The same answers as the floating-point comparisons in their comments, NaN
// included, from the bit patterns (on the integer pipe).
// v > 0
__device__ __forceinline__ bool is_positive(double v) { return dbits(v) - 1ull < 0x7FF0000000000000ull; }
// v > -1
__device__ __forceinline__ bool gt_minus_one(double v) {
  const uint64_t b = dbits(v);
  return (b >> 63) ? (abs_bits(v) < 0x3FF0000000000000ull) : (b <= 0x7FF0000000000000ull);
}
// v > -1 && v < inf
__device__ __forceinline__ bool in_minus_one_inf(double v) {
  const uint64_t b = dbits(v);
  return (b >> 63) ? (abs_bits(v) < 0x3FF0000000000000ull) : (b < 0x7FF0000000000000ull);
}
// |v| < 1
__device__ __forceinline__ bool abs_lt_one(double v) { return abs_bits(v) < 0x3FF0000000000000ull; }
// |v| >= 1/4
__device__ __forceinline__ bool abs_ge_quarter(double v) {
  return abs_bits(v) - 0x3FD0000000000000ull <= 0x7FF0000000000000ull - 0x3FD0000000000000ull;
}

// ---------------------------------------------------------------------------
// Particle state in registers.  opd = 1+delta, dm1 = (1+delta)^2 - 1,
// rv0v = 1/rvv and ep = 1 + beta0 ptau are derived from the stored state,
// and so are the drift's iep = 1/ep, iep2 = 1/ep^2 and
// c0 = ((1+delta)^2 - ep^2)/ep^2 = dm1/(gamma0^2 ep^2), and the thick maps'
// dmb = delta - beta0 ptau = dm1/(gamma0^2 ((1+delta) + ep)), written without
// the cancellation of delta against beta0 ptau.  Each instantiation keeps in
// registers only those it uses.
struct Part {
  double x, px, y, py, zeta, delta, ptau, rpp, rvv;
  double opd, dm1, rv0v, ep, epm1;  // epm1 = beta0 ptau (= ep - 1)
  double iep, iep2, c0, dmb;
  // quantum emission left to the warp (track_tile): photon count, curvature, gamma
  int em_k;
  double em_h, em_g;
};

__device__ __forceinline__ void derive_drift(Part& p, const RefDev& r) {
  p.iep = p.rvv * p.rpp;
  p.iep2 = p.iep * p.iep;
  const double g = p.dm1 * r.ig02;
  p.c0 = g * p.iep2;
  p.dmb = g / (p.opd + p.ep);
}

// ep = 1 + beta0 ptau (= opd / rvv), rv0v = 1/rvv = ep rpp
__device__ __forceinline__ void derive(Part& p, const RefDev& r) {
  p.opd = 1.0 + p.delta;
  p.dm1 = p.delta * (p.delta + 2.0);
  p.ep = fma(r.beta0, p.ptau, 1.0);
  p.rv0v = p.ep * p.rpp;
  p.epm1 = r.beta0 * p.ptau;
  derive_drift(p, r);
}

// (1+delta)^2 = 1 + 2 ptau/beta0 + ptau^2 = 1 + u in the form
// delta = u/(s+1), s = sqrt(1+u) = 1+delta; rpp = 1/s and rvv = s/ep.  The
// three quotients share one division, q = 1/(s (s+1) ep).
__device__ __forceinline__ void energy_update(Part& p, const RefDev& r) {
  const double u = p.ptau * (p.ptau + r.twoib0);
  const double s = sqrt(1.0 + u);
  const double a = s + 1.0;
  p.ep = fma(r.beta0, p.ptau, 1.0);
  const double sa = s * a;
  const double q = 1.0 / (sa * p.ep);
  p.delta = (u * (s * p.ep)) * q;
  p.opd = 1.0 + p.delta;
  p.dm1 = p.delta * (p.delta + 2.0);
  p.rpp = (a * p.ep) * q;
  p.rvv = (s * sa) * q;
  p.rv0v = p.ep * p.rpp;
  p.epm1 = r.beta0 * p.ptau;
  derive_drift(p, r);
}

__device__ __forceinline__ void apply_energy_loss(Part& p, double dpt, const RefDev& r) {
  const double rpp_old = p.rpp;
  p.ptau = p.ptau + dpt;
  energy_update(p, r);
  const double f = p.opd * rpp_old;
  p.px = p.px * f;
  p.py = p.py * f;
}

// Sine (shift 0) or cosine (shift 1): Cody-Waite reduction by pi/2 (three-part
// constant, round-to-nearest by the 1.5*2^52 shift), the quadrant advanced by
// `shift`, and the Taylor series of sin / cos on |r| <= pi/4.
__device__ __forceinline__ double trig_cw(double x, const SinTab& t, int shift) {
  const double P1 = 1.5707963267948965579989817342720925807952880859375;
  const double P2 = 6.123233995736766035868820147291818682e-17;
  const double P3 = -1.4973849048591698329435081771059e-33;
  const double TOP = 0.63661977236758134307553505349005744813783858296183;
  const double SH = 6755399441055744.0;
  const double k = (x * TOP + SH) - SH;
  double r = fma(-k, P1, x);
  r = fma(-k, P2, r);
  r = fma(-k, P3, r);
  const int q = (int)(((long long)k + shift) & 3);
  const double z = r * r;
  double res;
  if (q & 1) {
    double pc = t.c[10];
#pragma unroll
    for (int i = 9; i >= 0; i--) pc = fma(pc, z, t.c[i]);
    res = pc;
  } else {
    double ps = t.s[9];
#pragma unroll
    for (int i = 8; i >= 1; i--) ps = fma(ps, z, t.s[i]);
    res = fma(r * z, ps, r);
  }
  return (q & 2) ? -res : res;
}
__device__ __forceinline__ double sin_cw(double x, const SinTab& t) { return trig_cw(x, t, 0); }

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11) and the photon sampler.
// The four words of the current Philox block wait in b0..b3 and are handed
// out in that order by shifting the queue, so that every index is static and
// the block stays in registers (an indexed array would live in local memory).
struct Uni {
  uint64_t c0, c1, c2, c3, key;
  uint64_t b0, b1, b2, b3;
  int pos;
};
__device__ __forceinline__ void philox4x64(uint64_t& c0, uint64_t& c1, uint64_t& c2, uint64_t& c3,
                                           uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    const uint64_t hi0 = __umul64hi(m0, c0), lo0 = m0 * c0;
    const uint64_t hi1 = __umul64hi(m1, c2), lo1 = m1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}
// The next 64-bit Philox word; its uniform is (w >> 11) 2^-53 (unit53).
__device__ __forceinline__ uint64_t uni_word(Uni& u) {
  if (u.pos == 4) {
    uint64_t a = u.c0, b = u.c1, c = u.c2, d = u.c3;
    philox4x64(a, b, c, d, u.key, 0ull);
    u.b0 = a; u.b1 = b; u.b2 = c; u.b3 = d;
    u.c3 += 1;
    u.pos = 0;
  }
  const uint64_t w = u.b0;
  u.b0 = u.b1;
  u.b1 = u.b2;
  u.b2 = u.b3;
  u.pos++;
  return w;
}
// m 2^-53 for m < 2^53, assembled from its bits: the value is exact, the same
// as converting m and multiplying by 2^-53, but takes no FP64 instruction.
__device__ __forceinline__ double unit53(uint64_t m) {
  if (m == 0) return 0.0;
  const int e = 63 - __clzll((long long)m);  // leading bit, 0..52
  const uint64_t mant = (m << (52 - e)) & 0x000FFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(((uint64_t)(e + 970) << 52) | mant));  // exponent e - 53
}
// Inverse CDF of the photon spectrum: power-law asymptote F ~ xi^(1/3) below
// the first knot, clamp above the last, else linear interpolation on the
// knot interval [lo, lo+1] with lo = max{i : F[i] <= u}, found by walking up
// from the guide table's entry for u's cell of width 1/XT_SPEC_GUIDE.  F
// holds the K knots, then 1/(F[k+1] - F[k]) per interval and 1/F[0].
// u = (w >> 11) 2^-53 from the Philox word w.  u and the knots F are
// non-negative, so their order is the order of their bit patterns, and the
// comparisons run on the integer pipe; u's guide cell floor(u 4096) is w >> 52.
static_assert(XT_SPEC_GUIDE == 4096, "the guide cell is the top 12 bits of the Philox word");
__device__ __forceinline__ double sample_xi(uint64_t w, const double* xi, const double* F, const int32_t* guide,
                                            int K) {
  const double u = unit53(w >> 11);
  const uint64_t ub = dbits(u);
  if (ub < dbits(__ldg(F))) {
    const double q = u * __ldg(F + 2 * K);
    return __ldg(xi) * q * q * q;
  }
  if (ub >= dbits(__ldg(F + K - 1))) return __ldg(xi + K - 1);
  int lo = __ldg(guide + (int)(w >> 52));
  while (dbits(__ldg(F + lo + 1)) <= ub) lo++;
  const double f = (u - __ldg(F + lo)) * __ldg(F + K + lo);
  const double xl = __ldg(xi + lo);
  return xl + f * (__ldg(xi + lo + 1) - xl);
}

struct RadCtx {
  uint64_t seed;
  const double* xi;
  const double* F;
  const int32_t* guide;
  int K;
};

// ---------------------------------------------------------------------------
// Element maps.  `prm` points to the record's parameters in shared memory.

// (1+u)^(-1/2) - 1 by the Taylor series (Horner, dyadic coefficients) of
// order 3, 6 or 8, or by 1/sqrt(1+u) - 1.
__device__ __forceinline__ double inv_pz_m1_order3(double u) {
  double h = fma(-0.3125, u, 0.375);
  h = fma(h, u, -0.5);
  return h * u;
}
__device__ __forceinline__ double inv_pz_m1_order6(double u) {
  double h = fma(0.2255859375, u, -0.24609375);
  h = fma(h, u, 0.2734375);
  h = fma(h, u, -0.3125);
  h = fma(h, u, 0.375);
  h = fma(h, u, -0.5);
  return h * u;
}
__device__ __forceinline__ double inv_pz_m1_order8(double u) {
  double h = fma(0.196380615234375, u, -0.20947265625);
  h = fma(h, u, 0.2255859375);
  h = fma(h, u, -0.24609375);
  h = fma(h, u, 0.2734375);
  h = fma(h, u, -0.3125);
  h = fma(h, u, 0.375);
  h = fma(h, u, -0.5);
  return h * u;
}

// Exact drift, for the whole warp (dead lanes compute along and keep their
// coordinates).  With ep = 1 + beta0 ptau = (1+delta)/rvv, the square of the
// longitudinal momentum is pz^2 = ep^2 (1 + v), v = c0 - (px^2 + py^2)/ep^2,
// c0 = ((1+delta)^2 - ep^2)/ep^2 = dm1/(gamma0^2 ep^2).  Then
// yh = (1+v)^(-1/2) - 1 = ep/pz - 1 gives L/pz = (L/ep)(1 + yh) and the
// path-length term zeta += L (1 - ep/pz) = -L yh, formed from v, which holds
// only the transverse angles and delta/gamma0^2: no term cancels.  yh is the
// Taylor series of the lowest order whose truncation stays below half an ulp
// of yh on its interval -- order 3 for |v| <= 2^-18, 6 for |v| <= 2^-9, 8 for
// |v| <= 2^-7 -- else 1/sqrt(1+v) - 1.  The order is chosen per particle (so
// the result does not depend on the warp), but when all live lanes of the
// warp need the same order the warp branches to that series alone: a masked
// lane costs the FP64 pipe as much as an active one, so per-lane selection
// would issue every order's instructions.  Returns the loss code: -2 for a
// live lane whose v is not in (-1, inf) (pz not real), else 1 (dead lanes
// always 1).  The validity and order tests run on the integer pipe.
__device__ __forceinline__ int drift_warp(Part& p, const double* prm, bool alive) {
  const double L = prm[0];
  const double u = fma(-fma(p.px, p.px, p.py * p.py), p.iep2, p.c0);  // v
  const uint64_t ub = dbits(u), ua = abs_bits(u);
  const bool valid = (ub >> 63) ? (ua < 0x3FF0000000000000ull) : (ub < 0x7FF0000000000000ull);
  const bool run = alive && valid;
  const int tier = (ua <= 0x3ED0000000000000ull)   ? 1   // |u| <= 2^-18
                   : (ua <= 0x3F60000000000000ull) ? 2   // |u| <= 2^-9
                   : (ua <= 0x3F80000000000000ull) ? 3   // |u| <= 2^-7
                                                   : 4;
  const unsigned present = __reduce_or_sync(FULL_MASK, run ? (1u << tier) : 0u);
  if (present == 0) return (alive && !valid) ? -2 : 1;
  double yh;
  if (present == 2u) {
    yh = inv_pz_m1_order3(u);
  } else if (present == 4u) {
    yh = inv_pz_m1_order6(u);
  } else if (present == 8u) {
    yh = inv_pz_m1_order8(u);
  } else if (tier == 1) {
    yh = inv_pz_m1_order3(u);
  } else if (tier == 2) {
    yh = inv_pz_m1_order6(u);
  } else if (tier == 3) {
    yh = inv_pz_m1_order8(u);
  } else {
    yh = 1.0 / sqrt(1.0 + u) - 1.0;
  }
  if (run) {
    const double Li = L * p.iep;
    const double lpz = fma(Li, yh, Li);
    p.x = fma(p.px, lpz, p.x);
    p.y = fma(p.py, lpz, p.y);
    p.zeta = fma(-L, yh, p.zeta);
  }
  return (alive && !valid) ? -2 : 1;
}

// ---------------------------------------------------------------------------
// 4D beam-beam lens (section "Beam-beam interactions"): the transverse kick of
// a frozen Gaussian bunch.  Constant table from the host: [0] L, [1..40]
// Weideman's coefficients of the Faddeeva expansion, [41..59] 1/n!, and
// [60..73] the series coefficients of asin(v)/v (thick bend).
__constant__ double c_special[XT_SPECIAL_N];

// e^x: Cody-Waite reduction x = k ln2 + r (ln 2 as a 20-bit head, so that
// k * head is exact, plus a tail), e^r by its Taylor series to r^13 on
// |r| <= ln2/2, times 2^k from the exponent bits (two steps below the
// normal range).
// The range tests compare bit patterns on the integer pipe (745.2 and 709.7
// are 0x408749999999999A and 0x40862D999999999A); in range, s = x/ln2 + sh
// lies in [2^52, 2^53), where the integer k is the difference of the bits.
__device__ __forceinline__ double exp_cw(double x) {
  const uint64_t xb = dbits(x), xa = abs_bits(x);
  if (xa > 0x7FF0000000000000ull) return x;                          // NaN
  if (xb >> 63) {
    if (xa >= 0x408749999999999Aull) return 0.0;                       // x <= -745.2
  } else if (xa > 0x40862D999999999Aull) {
    return __longlong_as_double(0x7FF0000000000000ll);                 // x > 709.7
  }
  const double sh = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer
  const double s = fma(x, 1.4426950408889634, sh);
  const double t = s - sh;
  const int k = (int)(dbits(s) - dbits(sh));
  double r = fma(-t, 0x1.62e42p-1, x);
  r = fma(-t, 0x1.fdf473de6af28p-22, r);
  double p = c_special[41 + 13];
  for (int n = 12; n >= 0; n--) p = fma(p, r, c_special[41 + n]);
  if (k >= -1022) return p * __longlong_as_double((long long)(k + 1023) << 52);
  return (p * __longlong_as_double((long long)(k + 64 + 1023) << 52)) * __longlong_as_double((long long)(1023 - 64) << 52);
}

// 1 - e^(-u), u >= 0: the series u sum_n (-u)^n/(n+1)! below u = 1/2.
__device__ __forceinline__ double one_minus_exp(double u) {
  if (u < 0.5) {
    double s = c_special[41 + 18];
    for (int n = 16; n >= 0; n--) s = fma(s, -u, c_special[41 + n + 1]);
    return u * s;
  }
  return 1.0 - exp_cw(-u);
}

// w(x + i y), y >= 0: 2 p(Z) q^2 + q / sqrt(pi), q = 1/(L - i z),
// Z = (L + i z) q, given 1/D, D = |L - i z|^2 = (L + y)^2 + x^2 (so that the
// two evaluations of a lens share one division).
__device__ __forceinline__ void faddeeva_id(double x, double y, double iD, double* wr, double* wi) {
  const double L = c_special[0];
  const double cr = L + y;
  const double qr = cr * iD, qi = x * iD;
  const double ar = L - y;
  const double Zr = fma(ar, qr, -(x * qi));
  const double Zi = fma(ar, qi, x * qr);
  double pr = c_special[1 + 39], pi = 0.0;
  for (int n = 38; n >= 0; n--) {
    const double nr = fma(pr, Zr, fma(-pi, Zi, c_special[1 + n]));
    const double ni = fma(pr, Zi, pi * Zr);
    pr = nr;
    pi = ni;
  }
  const double tr = fma(pr, qr, -(pi * qi));
  const double ti = fma(pr, qi, pi * qr);
  const double ur = fma(2.0, tr, 0.5641895835477563);
  const double ui = 2.0 * ti;
  *wr = fma(qr, ur, -(qi * ui));
  *wi = fma(qr, ui, qi * ur);
}

// w at two points with one division: R = 1/(D1 D2), 1/D1 = D2 R, 1/D2 = D1 R
// (D is at least L^2, about 28, so the product cannot underflow).
__device__ __forceinline__ void faddeeva2(double x1, double y1, double x2, double y2, double* w1r, double* w1i,
                                          double* w2r, double* w2i) {
  const double L = c_special[0];
  const double c1 = L + y1, c2 = L + y2;
  const double D1 = fma(c1, c1, x1 * x1), D2 = fma(c2, c2, x2 * x2);
  const double R = 1.0 / (D1 * D2);
  faddeeva_id(x1, y1, D2 * R, w1r, w1i);
  faddeeva_id(x2, y2, D1 * R, w2r, w2i);
}

// Field shape of the unit bi-Gaussian line charge of record prm (K, x_c, y_c,
// mode, h1, h2, rs, rsi, 1/S, sqrt(pi)/S, lin1, lin2) at (x, y) about its
// centre.
__device__ __forceinline__ void bb_field(double x, double y, const double* prm, double* fx, double* fy) {
  const double ax = fabs(x), ay = fabs(y);
  const int mode = (int)prm[3];
  double gx, gy;
  if (mode == 0) {
    const double r2 = fma(ax, ax, ay * ay);
    const double g = (r2 == 0.0) ? prm[4] : one_minus_exp(r2 * prm[4]) / r2;
    gx = ax * g;
    gy = ay * g;
  } else {
    const double u = (mode == 1) ? ax : ay, v = (mode == 1) ? ay : ax;
    const double h = fma(u, u * prm[4], v * (v * prm[5]));
    double fu, fv;
    if (h < 5e-11) {
      fu = u * prm[10];
      fv = v * prm[11];
    } else {
      double w1r, w1i, w2r, w2i;
      faddeeva2(u * prm[8], v * prm[8], (u * prm[6]) * prm[8], (v * prm[7]) * prm[8], &w1r, &w1i, &w2r, &w2i);
      const double e = exp_cw(-h);
      fu = prm[9] * fma(-e, w2i, w1i);
      fv = prm[9] * fma(-e, w2r, w1r);
    }
    gx = (mode == 1) ? fu : fv;
    gy = (mode == 1) ? fv : fu;
  }
  *fx = copysign(gx, x);
  *fy = copysign(gy, y);
}

// Entire functions of z (either sign) with a = sqrt|z|: C = cos a,
// S = sin(a)/a, S2 = (1 - C)/z, S3 = (1 - S)/z for z > 0 (cosh and sinh for
// z < 0).  Series in z below |z| = 1, each to z^9 (1/n! from the special
// table), else from trig_cw or two exponentials.
__device__ __forceinline__ void osc_funcs(double z, const SinTab& sn, double* C, double* S, double* S2,
                                          double* S3) {
  if (abs_lt_one(z)) {
    const double mz = -z;
    const double* f = c_special + XT_SPECIAL_FACT;
    double c = f[18], s = f[19], s2 = f[20], s3 = f[21];
#pragma unroll
    for (int n = 8; n >= 0; n--) {
      c = fma(c, mz, f[2 * n]);
      s = fma(s, mz, f[2 * n + 1]);
      s2 = fma(s2, mz, f[2 * n + 2]);
      s3 = fma(s3, mz, f[2 * n + 3]);
    }
    *C = c; *S = s; *S2 = s2; *S3 = s3;
    return;
  }
  if (is_positive(z)) {
    const double a = sqrt(z);
    *C = trig_cw(a, sn, 1);
    *S = trig_cw(a, sn, 0) / a;
  } else {
    const double a = sqrt(-z);
    const double e = exp_cw(a), ei = exp_cw(-a);
    *C = 0.5 * (e + ei);
    *S = (0.5 * (e - ei)) / a;
  }
  *S2 = (1.0 - *C) / z;
  *S3 = (1.0 - *S) / z;
}

// asin(u)/u for |u| <= 1: the angle is halved, asin u = 2 asin v with
// v = u / sqrt(2 (1 + sqrt(1 - u^2))), until |v| < 1/4 (at most three times
// for |u| <= 1; the loop stops at four), then the series from the table.
__device__ __forceinline__ double asin_over(double u) {
  double v = u, m = 1.0;
  int halved = 0;
  for (; halved < 4 && abs_ge_quarter(v); halved++) {
    v = v / sqrt(2.0 * (1.0 + sqrt(1.0 - v * v)));
    m = m + m;
  }
  const double* a = c_special + XT_SPECIAL_ASIN;
  const double z = v * v;
  double s = a[13];
#pragma unroll
  for (int n = 12; n >= 0; n--) s = fma(s, z, a[n]);
  if (halved == 0) return s;
  return (m * (v / u)) * s;
}

// Thick bend, expanded model (section "Lattice modelling and single particle
// tracking": the model for large machines and small bending angles): the
// exact flow of
//   (px^2 + py^2) / (2 (1+delta)) - h x (1+delta) + k0 (x + h x^2 / 2) + k1 (x^2 - y^2) / 2,
// the curved-frame Hamiltonian with its square root expanded to second order
// in px, py.  x is a driven oscillator, px' = F - Kx x, F = h (1+delta) - k0,
// Kx = k0 h + k1; py' = k1 y; zeta' = 1 - (1/rvv)(1 + h x + (px^2 + py^2) /
// (2 (1+delta)^2)), integrated in closed form.  L of either sign.
__device__ __forceinline__ void bend_expanded(Part& p, double k0, double h, double L, double k1,
                                              const SinTab& sn) {
  const double Kx = k0 * h + k1, L2 = L * L;
  const double zx = (Kx * p.rpp) * L2;
  const double zy = ((-k1) * p.rpp) * L2;
  double C, S, S2, S3, Cy, Sy, S2y, S3y;
  osc_funcs(zx, sn, &C, &S, &S2, &S3);
  osc_funcs(zy, sn, &Cy, &Sy, &S2y, &S3y);
  const double x0 = p.x, px0 = p.px, y0 = p.y, py0 = p.py;
  const double F = fma(h, p.delta, h - k0);  // h (1+delta) - k0
  const double G = fma(-Kx, x0, F);
  const double Gy = k1 * y0;
  const double Lr = L * p.rpp;
  p.x = fma(C, x0, fma(Lr * S, px0, ((L * Lr) * S2) * F));
  p.px = fma(C, px0, (L * S) * G);
  p.y = fma(Cy, y0, (Lr * Sy) * py0);
  p.py = fma(Cy, py0, (L * Sy) * Gy);
  // integrals of x and of px^2 + py^2 over the body; (1 - C S)/z = S3 + S S2
  const double Ix = fma(L * S, x0, fma((L * Lr) * S2, px0, ((L2 * Lr) * S3) * F));
  const double hL = 0.5 * L, hL3 = 0.5 * (L2 * L);
  double I = (hL * fma(C, S, 1.0)) * (px0 * px0);
  I = fma(L2 * (S * S), px0 * G, I);
  I = fma(hL3 * fma(S, S2, S3), G * G, I);
  I = fma(hL * fma(Cy, Sy, 1.0), py0 * py0, I);
  I = fma(L2 * (Sy * Sy), py0 * Gy, I);
  I = fma(hL3 * fma(Sy, S2y, S3y), Gy * Gy, I);
  p.zeta = p.zeta + fma(L * p.dmb, p.rpp, -(p.rv0v * fma(h, Ix, (0.5 * (p.rpp * p.rpp)) * I)));
}

// Thick bend, full model (section "Lattice modelling and single particle
// tracking": the model for small machines): exact motion in a uniform field
// k0 through a sector of curvature h and length L (either sign).  From the
// invariants pX + k0 Z and pZ - k0 X of circular motion: at the exit plane
// px' = B - k0 (1/h + x) sin, x' = x cos - (1 - cos)/h + (1/h + x) sin
// (px' + B)/(pz' + Q), B = px cos + pz sin, Q = pz cos - px sin, with
// sin/h = L S and (1 - cos)/h = h L^2 S2 at z = (h L)^2; the horizontal arc
// length is chord * asin(u)/u, u = k0 chord / (2 p_h), and y, zeta follow it.
// Returns 1, or -2 (lost) if pz or pz' is not real or the exit plane is not
// reached.
// C, S, S2: the oscillator functions at z = (h L)^2 (from the record, or
// bend_full below for other lengths).
__device__ __forceinline__ int bend_full_c(Part& p, double k0, double h, double L, double C, double S,
                                           double S2) {
  const double th = h * L, L2 = L * L;
  const double snt = th * S, Sh = L * S, Ch = (h * L2) * S2, D2 = 2.0 * (L2 * S2);
  const double u = fma(-p.px, p.px, fma(-p.py, p.py, p.dm1));  // pz^2 - 1
  if (!in_minus_one_inf(u)) return -2;
  const double pz = sqrt(1.0 + u);
  const double ph2 = 1.0 + fma(-p.py, p.py, p.dm1);
  const double B = fma(p.px, C, pz * snt);
  const double Q = fma(pz, C, -(p.px * snt));
  const double r0s = fma(p.x, snt, Sh);  // (1/h + x) sin(theta)
  const double A = fma(-k0, r0s, B);     // px at the exit plane
  const double pzf2 = fma(-A, A, ph2);
  if (!is_positive(pzf2)) return -2;
  const double pzf = sqrt(pzf2);
  const double den = pzf + Q;
  if (!is_positive(den)) return -2;
  const double xf = fma(p.x, C, -Ch) + r0s * ((A + B) / den);
  const double dxf = xf - p.x;
  const double chord = sqrt(fma(dxf, dxf, (fma(h, p.x, 1.0) * fma(h, xf, 1.0)) * D2));
  const double ph = sqrt(ph2);
  const double uu = (k0 * chord) / (ph + ph);
  if (!abs_le_one(uu)) return -2;
  const double lh = ((L >= 0.0) ? chord : -chord) * asin_over(uu);
  const double lr = lh / ph;
  p.x = xf;
  p.px = A;
  p.y = fma(p.py, lr, p.y);
  p.zeta = p.zeta + fma(-p.ep, lr, L);
  return 1;
}
// Full-model bend with a gradient k1 (no closed form): n thin quadrupole
// kicks of strength k1 L/n between exact uniform-field bodies of lengths
// L/(2n), L/n, ..., L/n, L/(2n) -- drift-kick splitting, symplectic and of
// second order in L/n.  prm = k0, h, L, k1, C, S, S2 (whole body, unused
// here), n, C, S, S2 at z = (h L/(2n))^2, C, S, S2 at z = (h L/n)^2,
// L/(2n), L/n, k1 L/n.  sgn = -1 gives the inverse (the splitting is
// symmetric, so the same sequence with every length and kick negated).
__device__ __forceinline__ int bend_full_kicks(Part& p, const double* prm, double sgn) {
  const double k0 = prm[0], h = prm[1];
  const int n = (int)prm[7];
  const double lh = sgn * prm[14], ls = sgn * prm[15], kl = sgn * prm[16];
  int r = bend_full_c(p, k0, h, lh, prm[8], prm[9], prm[10]);
  for (int i = 0; i < n && r == 1; i++) {
    p.px = fma(-kl, p.x, p.px);
    p.py = fma(kl, p.y, p.py);
    r = (i + 1 < n) ? bend_full_c(p, k0, h, ls, prm[11], prm[12], prm[13])
                    : bend_full_c(p, k0, h, lh, prm[8], prm[9], prm[10]);
  }
  return r;
}

__device__ __forceinline__ int bend_full(Part& p, double k0, double h, double L, const SinTab& sn) {
  const double th = h * L;
  double C, S, S2, S3;
  osc_funcs(th * th, sn, &C, &S, &S2, &S3);
  return bend_full_c(p, k0, h, L, C, S, S2);
}

// Thick quadrupole (section "Lattice modelling and single particle tracking"):
// the exact flow, over a length L of either sign, of the expanded Hamiltonian
// (px^2 + py^2) / (2 (1+delta)) + k1 (x^2 - y^2) / 2.  Transverse motion is
// harmonic with w^2 = |k1| / (1+delta), cos / sin in the focusing plane (x when
// fx) and cosh / sinh in the other; zeta gains
// L (1 - 1/rvv) - (1 / (2 rvv (1+delta)^2)) * integral of (px^2 + py^2) ds,
// the integral in closed form.  C = cos a, Sa = sin(a)/a, Ch = cosh a and
// Sha = sinh(a)/a at a = w |L| are the oscillator functions at
// z = |k1| L^2 / (1+delta) and -z.
__device__ __forceinline__ void thick_quad(Part& p, double absk1, double L, bool fx, const SinTab& sn) {
  const double aK = absk1 * p.rpp;
  const double z = aK * (L * L);
  double C, Sa, Ch, Sha, u2, u3;
  osc_funcs(z, sn, &C, &Sa, &u2, &u3);
  osc_funcs(-z, sn, &Ch, &Sha, &u2, &u3);
  const double u0 = fx ? p.x : p.y, pu0 = fx ? p.px : p.py;
  const double v0 = fx ? p.y : p.x, pv0 = fx ? p.py : p.px;
  const double g = (aK * L) * Sa;    // w sin(w L)
  const double gh = (aK * L) * Sha;  // w sinh(w L)
  const double u1 = fma(C, u0, ((L * Sa) * p.rpp) * pu0);
  const double pu1 = fma(-(g * p.opd), u0, C * pu0);
  const double v1 = fma(Ch, v0, ((L * Sha) * p.rpp) * pv0);
  const double pv1 = fma(gh * p.opd, v0, Ch * pv0);
  const double o2 = p.opd * p.opd;
  const double A2 = pu0 * pu0, B2 = (aK * o2) * (u0 * u0);
  const double Ah2 = pv0 * pv0, Bh2 = (aK * o2) * (v0 * v0);
  const double hL = 0.5 * L;
  double I = hL * (A2 + B2);
  I = fma(hL * (Sa * C), A2 - B2, I);
  I = fma(-((p.opd * L) * (Sa * g)), pu0 * u0, I);
  I = fma(hL, Ah2 - Bh2, I);
  I = fma(hL * (Sha * Ch), Ah2 + Bh2, I);
  I = fma((p.opd * L) * (Sha * gh), pv0 * v0, I);
  // 1 - 1/rvv = (delta - beta0 ptau) / (1+delta)
  p.zeta = p.zeta + fma(L * p.dmb, p.rpp, -(((0.5 * p.rv0v) * (p.rpp * p.rpp)) * I));
  p.x = fx ? u1 : v1;
  p.px = fx ? pu1 : pv1;
  p.y = fx ? v1 : u1;
  p.py = fx ? pv1 : pu1;
}

// e^(-x) for the photon-count recurrence, x = nbar >= 0: x = j/64 + d with
// j = round(64 x) (the 1.5 * 2^52 shift; the integer read from the bits) and
// |d| <= 1/128, e^(-x) = E[j] e^(-d), E[j] = e^(-j/64) from the table that
// follows the spectrum's knots, e^(-d) by its Taylor series to d^7
// (truncation below 4e-19); x outside [0, 16) (or NaN) falls back to
// exp_cw, so the table index stays in 0..1024.
__device__ __forceinline__ double exp_neg(double x, const double* E) {
  if (!(x >= 0.0 && x < 16.0)) return exp_cw(-x);
  const double SH = 6755399441055744.0;
  const double t = fma(x, 64.0, SH);
  const int j = (int)(dbits(t) - dbits(SH));
  const double d = fma(-(t - SH), 0.015625, x);
  double e = fma(-d, 1.0 / 5040.0, 1.0 / 720.0);
  e = fma(e, -d, 1.0 / 120.0);
  e = fma(e, -d, 1.0 / 24.0);
  e = fma(e, -d, 1.0 / 6.0);
  e = fma(e, -d, 0.5);
  e = fma(e, -d, 1.0);
  e = fma(e, -d, 1.0);
  return __ldg(E + j) * e;
}

template <int RAD, bool DEFER = false>
__device__ __forceinline__ void multipole(Part& p, const double* prm, int order, int flags,
                                          const RefDev& r, const RadCtx& rc, int64_t pid, int turn,
                                          uint32_t elem) {
  const double2* cf = (const double2*)(prm + MP_COEF);
  const bool radiates = RAD != XT_RAD_OFF && (flags & REC_RAD);
  if (!radiates && (flags & (REC_PURE | REC_BEND))) {
    // last Horner step added straight into px, py; a bend's constant terms
    // combine to hxl * delta
    const bool bend = (flags & REC_BEND) != 0;
    double pxv = bend ? fma(prm[MP_HXL], p.delta, p.px) : p.px;
    if (order >= 1) {
      double2 c = cf[order];
      double ar = c.x, ai = c.y;
      for (int n = order - 1; n >= 1; n--) {
        c = cf[n];
        const double nr = fma(ar, p.x, fma(-ai, p.y, c.x));
        const double ni = fma(ar, p.y, fma(ai, p.x, c.y));
        ar = nr;
        ai = ni;
      }
      pxv = fma(-ar, p.x, fma(ai, p.y, pxv));
      p.py = fma(ar, p.y, fma(ai, p.x, p.py));
    }
    p.px = pxv;
    if (bend) {
      p.px = fma(-prm[MP_K0H], p.x, p.px);
      p.zeta = fma(-(prm[MP_HXL] * p.rv0v), p.x, p.zeta);
    }
    return;
  }
  // field of the orders >= 1, (fr, fi); the constant term c0 = (knl0, ksl0)
  // is added separately, and with a curvature the frame term hxl (1+delta)
  // joins -knl0 first, as (hxl - knl0) + hxl delta: in a ring's dipole slice
  // both are about 1e-3 while px is about 1e-5
  double fr = 0.0, fi = 0.0;
  if (order >= 1) {
    double2 c = cf[order];
    double ar = c.x, ai = c.y;
    for (int n = order - 1; n >= 1; n--) {
      c = cf[n];
      const double nr = fma(ar, p.x, fma(-ai, p.y, c.x));
      const double ni = fma(ar, p.y, fma(ai, p.x, c.y));
      ar = nr;
      ai = ni;
    }
    fr = fma(ar, p.x, -(ai * p.y));
    fi = fma(ar, p.y, ai * p.x);
  }
  const double2 c0 = cf[0];
  const double br = fr + c0.x, bi = fi + c0.y;
  p.py = p.py + bi;
  if (flags & REC_CURV) {
    const double hxl = prm[MP_HXL];
    p.px = (p.px - fr) + fma(hxl, p.delta, hxl - c0.x);
    p.px = fma(-prm[MP_K0H], p.x, p.px);
    p.zeta = fma(-(hxl * p.rv0v), p.x, p.zeta);
  } else {
    p.px = p.px - br;
  }
  if (RAD == XT_RAD_MEAN && (flags & REC_RAD)) {
    const double kk = fma(br, br, bi * bi);
    const double h2 = (kk * prm[MP_ILR2]) * (p.rpp * p.rpp);
    const double gam = fma(r.bg0, p.ptau, r.gamma0);
    const double bet = r.beta0 * p.rvv;
    const double b3 = bet * bet * bet;
    const double g2 = gam * gam;
    const double g4 = g2 * g2;
    const double dpt = (-prm[MP_CRL]) * b3 * g4 * h2;
    apply_energy_loss(p, dpt, r);
  } else if (RAD == XT_RAD_QUANTUM && (flags & REC_RAD)) {
    const double kk = fma(br, br, bi * bi);
    const double h = sqrt(kk * prm[MP_ILR2]) * p.rpp;
    const double gam = fma(r.bg0, p.ptau, r.gamma0);
    const double nbar = (prm[MP_KQL] * gam) * h;
    Uni u;
    u.c0 = (uint64_t)pid; u.c1 = (uint64_t)(uint32_t)turn; u.c2 = elem; u.c3 = 0;
    u.key = rc.seed; u.pos = 4;
    // k = min{k : u0 <= F_k} (at most 200), F_k = sum_{j<=k} e^-nbar nbar^j / j!,
    // decided first in FP32: F_k's FP32 value differs from its FP64 value
    // by less than 1e-5 for k <= 30 and nbar < 16 (expf and __fdividef within
    // 2 ulp, three roundings per step, nbar and u0 rounded to float), so
    // wherever u0 stays more than 2e-5 from every partial sum it passes, the
    // FP32 decision is the FP64 one.  Otherwise (or for larger k, nbar) the
    // FP64 recurrence decides, as below.
    const uint64_t w0 = uni_word(u);
    int k = 0;
    bool sure = nbar >= 0.0 && nbar < 16.0;
    if (sure) {
      const float nb = (float)nbar;
      const float u0f = __uint2float_rn((uint32_t)(w0 >> 40)) * 5.9604644775390625e-8f;  // top 24 bits / 2^24
      float pkf = expf(-nb), Ff = pkf;
      while (true) {
        const float gap = u0f - Ff;
        if (fabsf(gap) <= 2e-5f || k >= 30) {
          sure = false;
          break;
        }
        if (gap < 0.0f) break;
        k++;
        pkf = __fdividef(pkf * nb, (float)k);
        Ff = Ff + pkf;
      }
    }
    if (!sure) {
      // u0 and the partial sums F are non-negative (F is NaN only if nbar
      // is): the test u0 > F compares their bit patterns
      const uint64_t u0b = dbits(unit53(w0 >> 11));
      k = 0;
      double pk = exp_neg(nbar, rc.xi + rc.K), F = pk;
      while (u0b > dbits(F) && k < 200) {
        k++;
        pk = (pk * nbar) * c_special[XT_SPECIAL_RECIP + k];
        F = F + pk;
      }
    }
    if (DEFER) {  // the warp samples the photons together (emit_photons_warp)
      p.em_k = k;
      p.em_h = h;
      p.em_g = gam;
      return;
    }
    if (k > 0) {
      double sxi = 0.0;
      for (int j = 0; j < k; j++) sxi = sxi + sample_xi(uni_word(u), rc.xi, rc.F, rc.guide, rc.K);
      const double uc = (r.uc15 * (gam * gam * gam)) * h;
      const double dpt = -(uc * sxi) * r.ip0c;
      apply_energy_loss(p, dpt, r);
    }
  }
}

// Word idx (0-based) of the Philox stream of counter (c0, c1, c2): block
// idx / 4, position idx % 4, the order in which uni_word hands them out.
__device__ __forceinline__ uint64_t philox_word(uint64_t key, uint64_t c0, uint64_t c1, uint64_t c2, uint32_t idx) {
  uint64_t a = c0, b = c1, c = c2, d = (uint64_t)(idx >> 2);
  philox4x64(a, b, c, d, key, 0ull);
  const uint32_t q = idx & 3u;
  return q == 0 ? a : (q == 1 ? b : (q == 2 ? c : d));
}

// The photons of one radiating slice, sampled by the whole warp.  Every lane
// (lanes without photons, lost ones included, with em_k = 0) enters with its
// photon count; the warp's K photons are numbered by an exclusive prefix of
// the counts, and lane L samples photons L, L + 32, ...: photon j of owner o
// is word 1 + j of o's Philox stream (word 0 drew the count), so each value
// is the one the owner would draw itself.  The values go to this warp's
// XT_PHOTON_CAP doubles of shared memory, and each owner adds its own in the
// order j = 0, 1, ... -- the same sum, in the same order, as sampling them
// one by one, independent of which particles share the warp.  More than
// XT_PHOTON_CAP photons in the warp: every owner samples its own.
__device__ __forceinline__ void emit_photons_warp(Part& p, int64_t pid, int turn, uint32_t elem, const RadCtx& rc,
                                                  const RefDev& r, int lane, double* ph) {
  const int k = p.em_k;
  int incl = k;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(FULL_MASK, incl, off);
    if (lane >= off) incl += v;
  }
  const int K = __shfl_sync(FULL_MASK, incl, 31);
  if (K == 0) return;
  const int excl = incl - k;
  const uint64_t c1 = (uint64_t)(uint32_t)turn;
  double sxi = 0.0;
  if (K <= XT_PHOTON_CAP) {
    for (int base = 0; base < K; base += 32) {
      const int t = base + lane;
      // owner: the number of lanes whose inclusive count is <= t
      int o = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int v = __shfl_sync(FULL_MASK, incl, o + step - 1);
        if (v <= t) o += step;
      }
      const int os = o & 31;
      const int ex_o = __shfl_sync(FULL_MASK, excl, os);
      const int64_t pid_o = __shfl_sync(FULL_MASK, pid, os);
      if (t < K) {
        const uint64_t w = philox_word(rc.seed, (uint64_t)pid_o, c1, elem, (uint32_t)(1 + t - ex_o));
        ph[t] = sample_xi(w, rc.xi, rc.F, rc.guide, rc.K);
      }
    }
    __syncwarp();
    for (int j = 0; j < k; j++) sxi = sxi + ph[excl + j];
    __syncwarp();
  } else {
    Uni u;
    u.c0 = (uint64_t)pid; u.c1 = c1; u.c2 = elem; u.c3 = 0;
    u.key = rc.seed; u.pos = 4;
    uni_word(u);  // the count's word
    for (int j = 0; j < k; j++) sxi = sxi + sample_xi(uni_word(u), rc.xi, rc.F, rc.guide, rc.K);
  }
  if (k > 0) {
    const double gam = p.em_g;
    const double uc = (r.uc15 * (gam * gam * gam)) * p.em_h;
    const double dpt = -(uc * sxi) * r.ip0c;
    apply_energy_loss(p, dpt, r);
  }
}

// Dipole edge, non-linear model (section "Lattice modelling and single
// particle tracking": edge effects as full non-linear maps); prm = r21, r43,
// k0, t = tan(e), s (+1 entrance, -1 exit), corr.  The canonical map of the
// generating function x X' + y Y' + zeta Z' + (k0/2) y^2 T(px, py', delta)
// - (k0/2) t x^2 with T = tan(e + s atan(px/pz)) (the vertical kick of the
// fields a hard edge carries to first order in the field gradient): py' by
// fixed-point iteration until it stops changing (at most 40 steps), then x,
// y, zeta shifted by (k0/2) y^2 dT/d(px,
// py, pzeta); the wedge kick px += r21 x after it at the entrance, before it
// at the exit; the finite-extent correction py += corr y, corr = r21 + r43,
// so that the linearisation is the linear edge.  Returns -2 if pz is not real.
__device__ __forceinline__ int edge_nonlinear(Part& p, const double* prm) {
  const double r21 = prm[0], k0 = prm[2], t = prm[3], sgn = prm[4], corr = prm[5];
  if (sgn < 0.0) p.px = fma(r21, p.x, p.px);
  const double px = p.px, y = p.y, py = p.py;
  const double base = fma(-px, px, p.dm1);  // (1+delta)^2 - 1 - px^2
  if (!gt_minus_one(fma(-py, py, base))) return -2;
  const double ky = k0 * y;
  const double st = sgn * t;
  double pyn = py;
  for (int k = 0; k < 40; k++) {  // fixed-point iteration until py' no longer changes
    const double pz = sqrt(1.0 + fma(-pyn, pyn, base));
    const double Tv = fma(t, pz, sgn * px) / fma(-st, px, pz);
    const double nxt = fma(-ky, Tv, py);
    const bool same = nxt == pyn;
    pyn = nxt;
    if (same) break;
  }
  const double u = fma(-pyn, pyn, base);
  if (!gt_minus_one(u)) return -2;
  const double pz = sqrt(1.0 + u);
  const double D = fma(-st, px, pz);
  const double c = (sgn * (1.0 + t * t)) / (pz * (D * D));
  const double g = ((0.5 * k0) * (y * y)) * c;
  p.x = fma(g, fma(pz, pz, px * px), p.x);
  p.y = fma(g, px * pyn, p.y);
  p.zeta = fma(-(g * (px * p.opd)), p.rv0v, p.zeta);
  p.py = fma(corr, p.y, pyn);
  if (sgn > 0.0) p.px = fma(r21, p.x, p.px);
  return 1;
}

// Change of reference plane through a uniform vertical field k0 (k0 = 0:
// field-free): the new plane is the old one turned by the angle a (ca, sa)
// about the vertical axis through the reference point.  The particle starts
// at X = x ca, Z = -x sa of the new axes, with momenta px2 = px ca + pz sa,
// pzr = pz ca - px sa.  pX + k0 Z and pZ - k0 X are constant on its circle, so
// on the new plane px' = px2 - k0 x sa and x' = x ca + x sa (px2 + px')/(pz'
// + pzr); the direction turns by asin(k0 G/p_h^2), G = x sa (pzr + px2 (px2 +
// px')/(pz' + pzr)), and the path over p_h is lr = (G/p_h^2) asin(v)/v,
// v = k0 G/p_h^2; y += py lr, zeta -= ep lr.  Returns -2 if pz or pz' is not
// real or the plane is not reached.
__device__ __forceinline__ int plane_rot(Part& p, double k0, double ca, double sa) {
  const double ph2m1 = fma(-p.py, p.py, p.dm1);  // p_h^2 - 1
  const double u = fma(-p.px, p.px, ph2m1);      // pz^2 - 1
  if (!gt_minus_one(u)) return -2;
  const double pz = sqrt(1.0 + u);
  const double px2 = fma(p.px, ca, pz * sa);
  const double pzr = fma(pz, ca, -(p.px * sa));
  const double xs = p.x * sa;
  const double pxf = fma(-k0, xs, px2);
  const double uf = fma(-pxf, pxf, ph2m1);
  if (!gt_minus_one(uf)) return -2;
  const double den = sqrt(1.0 + uf) + pzr;
  if (!is_positive(den)) return -2;
  const double q = (px2 + pxf) / den;
  const double iph2 = 1.0 / (1.0 + ph2m1);
  const double G = xs * fma(px2, q, pzr);
  const double v = (k0 * G) * iph2;
  if (!abs_le_one(v)) return -2;
  const double lr = (G * iph2) * asin_over(v);
  p.x = fma(xs, q, p.x * ca);
  p.px = pxf;
  p.y = fma(p.py, lr, p.y);
  p.zeta = fma(-p.ep, lr, p.zeta);
  return 1;
}

// Dipole edge with the exact wedge: the non-linear fringe taken on the pole
// face (in its own frame, where the face angle is zero) between exact
// changes of plane.  Entrance: a straight line from the normal plane to the
// face (turned by e), the fringe, the field k0 back to the normal plane (-e);
// the exit is the mirror sequence.  prm = 0, r43, k0, 0, s (+1 entrance, -1
// exit), corr, cos e, sin e (edge_nonlinear reads the first six: no wedge
// kick, t = 0).
__device__ __forceinline__ int edge_wedge(Part& p, const double* prm) {
  const double k0 = prm[2], ce = prm[6], se = prm[7];
  const bool entrance = prm[4] > 0.0;
  int r = entrance ? plane_rot(p, 0.0, ce, se) : plane_rot(p, k0, ce, -se);
  if (r == 1) r = edge_nonlinear(p, prm);
  if (r == 1) r = entrance ? plane_rot(p, k0, ce, -se) : plane_rot(p, 0.0, ce, se);
  return r;
}

// One record.  Returns the loss code (1 = still alive).  THICK = false is the
// instantiation for tables without beam-beam lenses, thick quadrupoles,
// bends or non-linear edges (the host chooses it only for such tables): their
// bodies then stay out of the thin-element tracking loop.
template <int RAD, bool THICK = true, bool DEFER = false>
__device__ __forceinline__ int element(Part& p, uint32_t type, uint32_t order, uint32_t flags,
                                       uint32_t elem, const double* prm, const RefDev& r,
                                       const SinTab& sn, const RadCtx& rc, int64_t pid, int turn) {
  switch (type) {
    case XT_MULTIPOLE:
      multipole<RAD, DEFER>(p, prm, (int)order, (int)flags, r, rc, pid, turn, elem);
      return 1;
    case XT_APERTURE: {
      const double rr = fma(p.x, p.x, p.y * p.y);
      if (dbits(rr) > dbits(prm[0])) return (is_finite(p.x) && is_finite(p.y)) ? 0 : -1;
      return 1;
    }
    case XT_BEAMBEAM4D: {
      if constexpr (THICK) {
        double fx, fy;
        bb_field(p.x - prm[1], p.y - prm[2], prm, &fx, &fy);
        p.px = fma(prm[0], fx, p.px);
        p.py = fma(prm[0], fy, p.py);
      }
      return 1;
    }
    case XT_SPACECHARGE: {  // prm: K, centre, field constants, 1/(2 sigma_z^2) (0: coasting)
      if constexpr (THICK) {
        double fx, fy;
        bb_field(p.x - prm[1], p.y - prm[2], prm, &fx, &fy);
        const double g = (prm[12] > 0.0) ? exp_cw(-((p.zeta * p.zeta) * prm[12])) : 1.0;
        const double Kg = prm[0] * g;
        p.px = fma(Kg, fx, p.px);
        p.py = fma(Kg, fy, p.py);
      }
      return 1;
    }
    case XT_XYSHIFT:  // change of reference frame: displaced by (dx, dy)
      p.x = p.x - prm[0];
      p.y = p.y - prm[1];
      return 1;
    case XT_SROTATION: {  // change of reference frame: rotated about s (cos, sin)
      const double c = prm[0], sn = prm[1];
      const double x = p.x, y = p.y, px = p.px, py = p.py;
      p.x = fma(c, x, sn * y);
      p.y = fma(c, y, -(sn * x));
      p.px = fma(c, px, sn * py);
      p.py = fma(c, py, -(sn * px));
      return 1;
    }
    case XT_APERTURE_RECT: {
      const double x = p.x, y = p.y;
      if (!(x >= prm[0] && x <= prm[1] && y >= prm[2] && y <= prm[3]))
        return (is_finite(x) && is_finite(y)) ? 0 : -1;
      return 1;
    }
    case XT_APERTURE_ELLIPSE: {  // prm = 1/a^2, 1/b^2; t >= 0 or NaN, so its bits order it
      const double t = fma(p.x * p.x, prm[0], (p.y * p.y) * prm[1]);
      if (dbits(t) > 0x3FF0000000000000ull) return (is_finite(p.x) && is_finite(p.y)) ? 0 : -1;
      return 1;
    }
    case XT_CAVITY: {
      const double phi = fma(-prm[0], p.zeta, prm[1]);
      p.ptau = fma(prm[2], sin_cw(phi, sn), p.ptau);
      energy_update(p, r);
      return 1;
    }
    case XT_DIPEDGE:
      if constexpr (THICK) {
        if (flags & REC_EWEDGE) return edge_wedge(p, prm);
        if (flags & REC_ENL) return edge_nonlinear(p, prm);
      }
      p.px = fma(prm[0], p.x, p.px);
      p.py = fma(prm[1], p.y, p.py);
      return 1;
    case XT_QUAD:  // prm = |k1|, L; flags = REC_QF when x is the focusing plane
      if constexpr (THICK) thick_quad(p, prm[0], prm[1], (flags & REC_QF) != 0, sn);
      return 1;
    case XT_BEND:  // prm = k0, h, L, k1; flags = REC_BFULL for the full model
      if constexpr (THICK) {
        if (flags & REC_BKICK) return bend_full_kicks(p, prm, 1.0);
        if (flags & REC_BFULL) return bend_full_c(p, prm[0], prm[1], prm[2], prm[4], prm[5], prm[6]);
        bend_expanded(p, prm[0], prm[1], prm[2], prm[3], sn);
      }
      return 1;
    case XT_LINEARMAP: {
      const double v[6] = {p.x, p.px, p.y, p.py, p.zeta, p.ptau};
      double o[6];
#pragma unroll
      for (int i = 0; i < 6; i++) {
        double acc = prm[36 + i];
#pragma unroll
        for (int j = 0; j < 6; j++) acc = fma(prm[6 * i + j], v[j], acc);
        o[i] = acc;
      }
      p.x = o[0]; p.px = o[1]; p.y = o[2]; p.py = o[3]; p.zeta = o[4]; p.ptau = o[5];
      energy_update(p, r);
      return 1;
    }
    default:
      return 1;
  }
}

// ---------------------------------------------------------------------------
// The tile body shared by the single-lattice and the batched kernels.
struct TileLat {
  const uint8_t* lat;
  const Chunk* chunks;
  int nch;
  int n_el;
};
struct TileArrays {
  double *x, *px, *y, *py, *zeta, *delta, *ptau, *rpp, *rvv;
  int32_t *state, *at_turn, *at_element;
  const int64_t* pid;
};
struct Ctl {
  int32_t* status;
  const volatile int32_t* cancel;
  int64_t max_cycles;
  int64_t t_start;
  int64_t last_poll;
};

// Returns 0, or an XT_ERR_* code if the launch must stop (cancel, budget, staging).
template <int RAD, bool THICK>
__device__ __forceinline__ int track_tile(const TileLat& L, const TileArrays& A, int i, bool active, int turn0,
                          int n_turns, Stage& st, int& resident_key, int lat_key,
                          const RefDev& ref, const SinTab& sn, const RadCtx& rc, Ctl& ctl,
                          int lane, double* ph) {
  Part p;
  int code = 0, lturn = 0;
  uint32_t lelem = 0;
  int64_t pid = 0;
  if (active) {
    p.x = A.x[i]; p.px = A.px[i]; p.y = A.y[i]; p.py = A.py[i]; p.zeta = A.zeta[i];
    p.delta = A.delta[i]; p.ptau = A.ptau[i]; p.rpp = A.rpp[i]; p.rvv = A.rvv[i];
    code = A.state[i];
    pid = A.pid[i];
  } else {
    p.x = p.px = p.y = p.py = p.zeta = p.delta = p.ptau = 0.0;
    p.rpp = p.rvv = 1.0;
  }
  bool alive = active && code == 1;
  derive(p, ref);
  int err = 0;
  int done_turns = 0;
  const int nch = L.nch;
  const int64_t total = (int64_t)n_turns * nch;
  int64_t seq = 0;
  if (nch > 1) {
    resident_key = -1;  // buffer 0 is about to be overwritten
    stage_issue(st, 0, L.lat + L.chunks[0].off, L.chunks[0].bytes, lane);
    if (total > 1) stage_issue(st, 1, L.lat + L.chunks[1 % nch].off, L.chunks[1 % nch].bytes, lane);
  }
  for (int turn = turn0; turn < turn0 + n_turns; ++turn) {
    for (int c = 0; c < nch; ++c, ++seq) {
      const uint8_t* buf;
      const int b = (int)(seq & 1);
      if (nch == 1) {
        if (resident_key != lat_key) {
          stage_issue(st, 0, L.lat + L.chunks[0].off, L.chunks[0].bytes, lane);
          if (!stage_wait(st, 0)) { err = XT_ERR_CUDA; break; }
          resident_key = lat_key;
        }
        buf = st.buf[0];
      } else {
        if (!stage_wait(st, b)) { err = XT_ERR_CUDA; break; }
        buf = b ? st.buf[1] : st.buf[0];
      }
      const uint32_t nrec = __ldg(&L.chunks[c].nrec);
      const uint8_t* q = buf;
      for (uint32_t rr = 0; rr < nrec; ++rr) {
        const uint4 hv = *(const uint4*)q;
        const uint32_t type = hv.x & 0xFFFFu, order = hv.x >> 16;
        const uint32_t flags = hv.y & 0xFFFFu, size16 = hv.y >> 16;
        const double* prm = (const double*)(q + 16);
        int lc = 1;
        if (RAD == XT_RAD_QUANTUM) p.em_k = 0;
        if (type == XT_DRIFT) {
          lc = drift_warp(p, prm, alive);
        } else if (type == XT_APERTURE) {
          // inside the inscribed square (integer pipe) => inside the circle;
          // the FP64 test runs only if some live lane of the warp is outside
          const uint64_t box = dbits(prm[1]);
          const bool in = !alive || (abs_bits(p.x) <= box && abs_bits(p.y) <= box);
          if (!__all_sync(FULL_MASK, in) && alive) lc = element<RAD, THICK>(p, type, order, flags, hv.z, prm, ref,
                                                                      sn, rc, pid, turn);
        } else if (alive) {
          lc = element<RAD, THICK, RAD == XT_RAD_QUANTUM>(p, type, order, flags, hv.z, prm, ref, sn, rc, pid, turn);
        }
        // quantum emission of a radiating multipole: the whole warp samples
        // the photons its lanes drew (the record is the same for every lane)
        if (RAD == XT_RAD_QUANTUM && type == XT_MULTIPOLE && (flags & REC_RAD))
          emit_photons_warp(p, pid, turn, hv.z, rc, ref, lane, ph);
        if (lc != 1) {
          alive = false;
          code = lc;
          lturn = turn;
          lelem = hv.z;
        }
        q += size16 * 16u;
      }
      if (nch > 1) {
        __syncwarp();
        if (seq + 2 < total) {
          const int cn = (int)((seq + 2) % nch);
          stage_issue(st, b, L.lat + L.chunks[cn].off, L.chunks[cn].bytes, lane);
        }
      }
      if (!__any_sync(FULL_MASK, alive)) break;
    }
    if (err) break;
    if (alive && !(abs_le_one(p.x) && abs_le_one(p.y))) {
      alive = false;
      code = -3;
      lturn = turn;
      lelem = (uint32_t)(L.n_el - 1);
    }
    done_turns = turn - turn0 + 1;
    if (!__any_sync(FULL_MASK, alive)) break;
    // cancel flag and cycle budget, checked by lane 0 at most every POLL_INTERVAL
    int stop = 0;
    if (lane == 0) {
      const int64_t now = clock64();
      if (ctl.max_cycles > 0 && now - ctl.t_start > ctl.max_cycles) stop = XT_ERR_TIMEOUT;
      else if (now - ctl.last_poll > POLL_INTERVAL) {
        ctl.last_poll = now;
        if (*ctl.cancel) stop = XT_ERR_CANCELLED;
      }
    }
    stop = __shfl_sync(FULL_MASK, stop, 0);
    if (stop && turn + 1 < turn0 + n_turns) { err = stop; break; }
  }
  stage_drain(st);
  if (active) {
    A.x[i] = p.x; A.px[i] = p.px; A.y[i] = p.y; A.py[i] = p.py; A.zeta[i] = p.zeta;
    A.delta[i] = p.delta; A.ptau[i] = p.ptau; A.rpp[i] = p.rpp; A.rvv[i] = p.rvv;
    if (alive) {
      A.at_turn[i] = turn0 + done_turns;
      A.at_element[i] = 0;
    } else if (code != 1) {
      A.state[i] = code;
      A.at_turn[i] = lturn;
      A.at_element[i] = (int32_t)lelem;
    }
  }
  return err;
}

// This warp's XT_PHOTON_CAP doubles after the chunk buffers (allocated by
// the host for the quantum-radiation kinds only; see track_smem_bytes).
__device__ __forceinline__ double* photon_buffer(uint8_t* smem, int chunk_bytes) {
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint8_t* end = smem + ((nwarps * 16 + 127) & ~127) + (size_t)nwarps * 2 * chunk_bytes;
  return (double*)end + (size_t)warp * XT_PHOTON_CAP;
}

__device__ __forceinline__ void stage_setup(Stage& st, uint8_t* smem, int chunk_bytes, int lane) {
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint64_t* bars = (uint64_t*)smem;
  uint8_t* bufs = smem + ((nwarps * 16 + 127) & ~127);
  st.buf[0] = bufs + (size_t)warp * 2 * chunk_bytes;
  st.buf[1] = st.buf[0] + chunk_bytes;
  st.bar[0] = bars + 2 * warp;
  st.bar[1] = bars + 2 * warp + 1;
  st.parity = 0;
  st.pending = 0;
  if (lane == 0) {
    mbar_init(st.bar[0], 1);
    mbar_init(st.bar[1], 1);
    fence_mbar_init();
  }
  __syncwarp();
}

__device__ __forceinline__ void set_status(int32_t* status, int err) {
  if (err) atomicCAS(status, 0, err);
}

// KIND = radiation mode + 3 if the table has thick rows (see element()).
// The thin instantiations without quantum radiation (KIND 0, 1) ask for 3
// blocks of XT_MAX_BLOCK per SM, which caps them at 80 registers with no
// spills; the quantum and thick ones (KIND >= 2) ask for 2, which lets their
// long paths run without spill code (measured +0.6 % to +0.7 %).
template <int KIND>
__global__ void __launch_bounds__(XT_MAX_BLOCK, (KIND >= 2) ? 2 : 3) track_kernel(const TrackArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  Stage st;
  stage_setup(st, smem, a.chunk_bytes, lane);
  double* const ph = photon_buffer(smem, a.chunk_bytes);
  if (*(volatile int32_t*)a.status != 0) return;
  const int n_alive = *a.n_alive;
  const TileLat L = {a.lat, a.chunks, a.n_chunks, a.n_el};
  const TileArrays A = {a.x, a.px, a.y, a.py, a.zeta, a.delta, a.ptau, a.rpp, a.rvv,
                        a.state, a.at_turn, a.at_element, a.pid};
  const RadCtx rc = {a.seed, a.spec_xi, a.spec_F, a.spec_guide, a.spec_k};
  Ctl ctl = {a.status, a.cancel, a.max_cycles, clock64(), clock64()};
  int resident = -1;
  // First tile: warp j of block b takes tile j * gridDim.x + b, so that when
  // there are fewer tiles than warps they spread evenly over the blocks and
  // hence the SMs; later tiles come from the queue, after the first round.
  const int first_round = gridDim.x * (blockDim.x >> 5);
  int tile = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  for (;; ) {
    const int64_t base = (int64_t)tile * 32;
    if (base >= n_alive) break;
    const int64_t k = base + lane;
    const bool active = k < n_alive;
    const int i = active ? __ldg(a.idx + k) : 0;
    const int err = track_tile<KIND % 3, (KIND >= 3)>(L, A, i, active, a.turn0, a.n_turns, st, resident, 0,
                                                     a.ref, a.sn, rc, ctl, lane, ph);
    if (err) {
      if (lane == 0) set_status(a.status, err);
      break;
    }
    int t = 0;
    if (lane == 0) t = first_round + atomicAdd(a.tile_counter, 1);
    tile = __shfl_sync(FULL_MASK, t, 0);
  }
}

template <int KIND>
__global__ void __launch_bounds__(XT_MAX_BLOCK, (KIND >= 2) ? 2 : 3) track_batched_kernel(const BatchArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  Stage st;
  stage_setup(st, smem, a.chunk_bytes, lane);
  double* const ph = photon_buffer(smem, a.chunk_bytes);
  if (*(volatile int32_t*)a.status != 0) return;
  const int64_t total_tiles = a.tile_prefix[a.n_seeds];
  const int turn0 = *a.turn_base + a.turn_off;
  const RadCtx rc = {a.seed, a.spec_xi, a.spec_F, a.spec_guide, a.spec_k};
  Ctl ctl = {a.status, a.cancel, a.max_cycles, clock64(), clock64()};
  int resident = -1;
  // first tile interleaved over the blocks, as in track_kernel
  const int first_round = gridDim.x * (blockDim.x >> 5);
  int tile = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  for (;; ) {
    if ((int64_t)tile >= total_tiles) break;
    // seed j in processing order with tile_prefix[j] <= tile < tile_prefix[j+1]
    int lo = 0, hi = a.n_seeds;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.tile_prefix[mid] <= tile) lo = mid; else hi = mid;
    }
    const int s = a.seed_order[lo];
    const SeedDev& S = a.seeds[s];
    const int64_t k = ((int64_t)tile - a.tile_prefix[lo]) * 32 + lane;
    const int nal = a.n_alive[s];
    const bool active = k < nal;
    const int i = active ? __ldg(a.idx + a.idx_base[s] + k) : 0;
    const TileLat L = {S.lat, S.chunks, S.n_chunks, S.n_el};
    const TileArrays A = {S.x, S.px, S.y, S.py, S.zeta, S.delta, S.ptau, S.rpp, S.rvv,
                          S.state, S.at_turn, S.at_element, S.pid};
    const int err = track_tile<KIND % 3, (KIND >= 3)>(L, A, i, active, turn0, a.n_turns, st, resident, s,
                                                     a.ref, a.sn, rc, ctl, lane, ph);
    if (err) {
      if (lane == 0) set_status(a.status, err);
      break;
    }
    int t = 0;
    if (lane == 0) t = first_round + atomicAdd(a.tile_counter, 1);
    tile = __shfl_sync(FULL_MASK, t, 0);
  }
}

// ---------------------------------------------------------------------------
// Loss-location refinement (section "Particle-matter interaction and
// collimation studies"): one thread per lost particle, backtracking to the
// previous aperture with the inverse maps, then re-tracking with drifts cut
// into steps and each step end tested against the aperture polygon
// interpolated in s.  Particles sit at different places, so there are no
// warp votes here: the series order of the drift is chosen per lane.

__device__ __forceinline__ bool drift_lane(Part& p, double L) {
  const double u = fma(-fma(p.px, p.px, p.py * p.py), p.iep2, p.c0);  // v, as in drift_warp
  const uint64_t ub = dbits(u), ua = abs_bits(u);
  const bool valid = (ub >> 63) ? (ua < 0x3FF0000000000000ull) : (ub < 0x7FF0000000000000ull);
  if (!valid) return false;
  double yh;
  if (ua <= 0x3ED0000000000000ull) yh = inv_pz_m1_order3(u);
  else if (ua <= 0x3F60000000000000ull) yh = inv_pz_m1_order6(u);
  else if (ua <= 0x3F80000000000000ull) yh = inv_pz_m1_order8(u);
  else yh = 1.0 / sqrt(1.0 + u) - 1.0;
  const double Li = L * p.iep;
  const double lpz = fma(Li, yh, Li);
  p.x = fma(p.px, lpz, p.x);
  p.y = fma(p.py, lpz, p.y);
  p.zeta = fma(-L, yh, p.zeta);
  return true;
}

// Inverse of one record's map, radiation off.  False if there is none here
// (linear map) or the backward drift is not defined.
__device__ __forceinline__ bool inverse_record(Part& p, uint32_t type, uint32_t order, uint32_t flags,
                                               const double* prm, const RefDev& r, const SinTab& sn) {
  switch (type) {
    case XT_DRIFT: return drift_lane(p, -prm[0]);
    case XT_MULTIPOLE: {  // x, y are unchanged by the kick: recompute the field, take it back
      const double2* cf = (const double2*)(prm + MP_COEF);
      double fr = 0.0, fi = 0.0;
      if (order >= 1) {
        double2 c = cf[order];
        double ar = c.x, ai = c.y;
        for (int n = (int)order - 1; n >= 1; n--) {
          c = cf[n];
          const double nr = fma(ar, p.x, fma(-ai, p.y, c.x));
          const double ni = fma(ar, p.y, fma(ai, p.x, c.y));
          ar = nr;
          ai = ni;
        }
        fr = fma(ar, p.x, -(ai * p.y));
        fi = fma(ar, p.y, ai * p.x);
      }
      const double2 c0 = cf[0];
      p.py = p.py - (fi + c0.y);
      if (flags & REC_CURV) {
        const double hxl = prm[MP_HXL];
        p.zeta = fma(hxl * p.rv0v, p.x, p.zeta);
        p.px = fma(prm[MP_K0H], p.x, p.px);
        p.px = (p.px + fr) - fma(hxl, p.delta, hxl - c0.x);
      } else {
        p.px = p.px + (fr + c0.x);
      }
      return true;
    }
    case XT_CAVITY: {
      const double phi = fma(-prm[0], p.zeta, prm[1]);
      p.ptau = fma(-prm[2], sin_cw(phi, sn), p.ptau);
      energy_update(p, r);
      return true;
    }
    case XT_DIPEDGE:
      if (flags & REC_ENL) return false;  // no inverse formed for the non-linear edges
      p.px = fma(-prm[0], p.x, p.px);
      p.py = fma(-prm[1], p.y, p.py);
      return true;
    case XT_QUAD:
      thick_quad(p, prm[0], -prm[1], (flags & REC_QF) != 0, sn);
      return true;
    case XT_BEND:
      if (flags & REC_BKICK) return bend_full_kicks(p, prm, -1.0) == 1;
      if (flags & REC_BFULL) return bend_full_c(p, prm[0], prm[1], -prm[2], prm[4], prm[5], prm[6]) == 1;
      bend_expanded(p, prm[0], prm[1], -prm[2], prm[3], sn);
      return true;
    case XT_LINEARMAP: return false;
    case XT_BEAMBEAM4D: {  // x, y unchanged by the kick: take the same kick back
      double fx, fy;
      bb_field(p.x - prm[1], p.y - prm[2], prm, &fx, &fy);
      p.px = fma(-prm[0], fx, p.px);
      p.py = fma(-prm[0], fy, p.py);
      return true;
    }
    case XT_SPACECHARGE: {  // x, y, zeta unchanged by the kick: take the same kick back
      double fx, fy;
      bb_field(p.x - prm[1], p.y - prm[2], prm, &fx, &fy);
      const double g = (prm[12] > 0.0) ? exp_cw(-((p.zeta * p.zeta) * prm[12])) : 1.0;
      const double Kg = prm[0] * g;
      p.px = fma(-Kg, fx, p.px);
      p.py = fma(-Kg, fy, p.py);
      return true;
    }
    case XT_XYSHIFT:
      p.x = p.x + prm[0];
      p.y = p.y + prm[1];
      return true;
    case XT_SROTATION: {
      const double c = prm[0], s = prm[1];
      const double x = p.x, y = p.y, px = p.px, py = p.py;
      p.x = fma(c, x, -(s * y));
      p.y = fma(c, y, s * x);
      p.px = fma(c, px, -(s * py));
      p.py = fma(c, py, s * px);
      return true;
    }
    default: return true;  // apertures
  }
}

// Crossing-number test of (x, y) against the polygon interpolated at weight
// w between polygons A and B (n vertices, x then y per vertex).
__device__ __forceinline__ bool inside_polygon(double x, double y, const double* A, const double* B, double w,
                                               int n) {
  bool in = false;
  for (int k = 0; k < n; k++) {
    const int k2 = (k + 1 == n) ? 0 : k + 1;
    const double ax = fma(w, B[2 * k] - A[2 * k], A[2 * k]);
    const double ay = fma(w, B[2 * k + 1] - A[2 * k + 1], A[2 * k + 1]);
    const double bx = fma(w, B[2 * k2] - A[2 * k2], A[2 * k2]);
    const double by = fma(w, B[2 * k2 + 1] - A[2 * k2 + 1], A[2 * k2 + 1]);
    if ((ay > y) != (by > y)) {
      const double xi = ax + (y - ay) * (bx - ax) / (by - ay);
      if (x < xi) in = !in;
    }
  }
  return in;
}

__global__ void __launch_bounds__(128) refine_kernel(RefineArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  a.s_loss[i] = nan;
  const int e = a.at_element[i];
  if (a.state[i] != 0 || e < 0 || e >= a.n_el) return;
  const int q = a.prev_ap[e];
  if (q < 0 || a.poly_idx[e] < 0 || a.poly_idx[q] < 0) return;
  Part p;
  p.x = a.x[i]; p.px = a.px[i]; p.y = a.y[i]; p.py = a.py[i]; p.zeta = a.zeta[i];
  p.delta = a.delta[i]; p.ptau = a.ptau[i]; p.rpp = a.rpp[i]; p.rvv = a.rvv[i];
  derive(p, a.ref);
  for (int j = e;;) {  // back to the exit of q
    j = (j == 0) ? a.n_el - 1 : j - 1;
    if (j == q) break;
    const int off = a.row_off[j];
    if (off < 0) continue;
    const uint4 hv = *(const uint4*)(a.lat + off);
    if (!inverse_record(p, hv.x & 0xFFFFu, hv.x >> 16, hv.y & 0xFFFFu, (const double*)(a.lat + off + 16), a.ref,
                        a.sn))
      return;
  }
  const double* PA = a.polys + (int64_t)a.poly_idx[q] * 2 * a.n_angles;
  const double* PB = a.polys + (int64_t)a.poly_idx[e] * 2 * a.n_angles;
  const double s_q = a.spos[q];
  const double C = a.spos[a.n_el];
  const double seg = (e > q) ? a.spos[e] - s_q : a.spos[e] + C - s_q;
  double pos = s_q;
  double found = nan;
  bool hit = false;
  RadCtx rc;
  rc.seed = 0; rc.xi = nullptr; rc.F = nullptr; rc.guide = nullptr; rc.K = 0;
  for (int j = q;;) {
    j = (j + 1 == a.n_el) ? 0 : j + 1;
    if (j == e) break;
    const int off = a.row_off[j];
    if (off < 0) continue;
    const uint4 hv = *(const uint4*)(a.lat + off);
    const uint32_t type = hv.x & 0xFFFFu;
    const double* prm = (const double*)(a.lat + off + 16);
    // drifts, thick quadrupoles and thick bends in steps of at most ds (the
    // thick maps are flows: their steps compose to the same map as one pass;
    // a full bend with kicks is not, and is passed whole)
    const double L = (type == XT_DRIFT) ? prm[0] : (type == XT_QUAD) ? prm[1] : (type == XT_BEND) ? prm[2] : 0.0;
    const bool kicked = type == XT_BEND && ((hv.y & 0xFFFFu) & REC_BKICK);
    if ((type == XT_DRIFT || type == XT_QUAD || type == XT_BEND) && L > 0.0 && !kicked) {
      const int64_t ns = (int64_t)ceil(L / a.ds);
      const double h = L / (double)ns;
      const double c = a.frame[4 * j], sn = a.frame[4 * j + 1], dx = a.frame[4 * j + 2], dy = a.frame[4 * j + 3];
      const uint32_t fl = hv.y & 0xFFFFu;
      for (int64_t k = 1; k <= ns; k++) {
        bool ok = true;
        if (type == XT_QUAD) thick_quad(p, prm[0], h, (fl & REC_QF) != 0, a.sn);
        else if (type == XT_BEND && (fl & REC_BFULL)) ok = bend_full(p, prm[0], prm[1], h, a.sn) == 1;
        else if (type == XT_BEND) bend_expanded(p, prm[0], prm[1], h, prm[3], a.sn);
        else ok = drift_lane(p, h);
        const double at = fma((double)k, h, pos);
        if (!ok) { found = at; hit = true; break; }
        const double lx = (c * p.x - sn * p.y) + dx;
        const double ly = (sn * p.x + c * p.y) + dy;
        const double w = (at - s_q) / seg;
        if (!inside_polygon(lx, ly, PA, PB, w, a.n_angles)) { found = at; hit = true; break; }
      }
      if (hit) break;
      pos = pos + L;
    } else if (type == XT_DRIFT) {
      if (!drift_lane(p, prm[0])) { found = pos; hit = true; break; }
    } else if (element<XT_RAD_OFF>(p, type, hv.x >> 16, hv.y & 0xFFFFu, hv.z, prm, a.ref, a.sn, rc, 0, 0) != 1) {
      found = pos;
      hit = true;
      break;
    } else if (kicked) {
      pos = pos + L;
    }
  }
  if (!hit) found = a.spos[e];
  a.s_loss[i] = (found >= C) ? found - C : found;
}

// ---------------------------------------------------------------------------
// Monitor: one pass of the table with the particle state written after every
// row (for lattice functions along the line and the tapering loop).  The maps,
// the loss rules and the end-of-turn guard are those of the tracking kernel,
// so the final state equals one turn of xt_track bit for bit.
template <int RAD>
__global__ void __launch_bounds__(128) monitor_kernel(const MonitorArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  Part p;
  p.x = a.x[i]; p.px = a.px[i]; p.y = a.y[i]; p.py = a.py[i]; p.zeta = a.zeta[i];
  p.delta = a.delta[i]; p.ptau = a.ptau[i]; p.rpp = a.rpp[i]; p.rvv = a.rvv[i];
  int code = a.state[i];
  const int64_t pid = a.pid[i];
  bool alive = code == 1;
  int lturn = a.at_turn[i];
  int lelem = a.at_element[i];
  derive(p, a.ref);
  const RadCtx rc = {a.seed, a.spec_xi, a.spec_F, a.spec_guide, a.spec_k};
  const int64_t n = a.n;
  for (int r = 0; r < a.n_el; r++) {
    const int off = a.row_off[r];
    if (off >= 0 && alive) {
      const uint4 hv = *(const uint4*)(a.lat + off);
      const uint32_t type = hv.x & 0xFFFFu;
      const double* prm = (const double*)(a.lat + off + 16);
      int lc;
      if (type == XT_DRIFT) lc = drift_lane(p, prm[0]) ? 1 : -2;
      else lc = element<RAD>(p, type, hv.x >> 16, hv.y & 0xFFFFu, hv.z, prm, a.ref, a.sn, rc, pid, a.turn);
      if (lc != 1) {
        alive = false;
        code = lc;
        lturn = a.turn;
        lelem = (int)hv.z;
      }
    }
    if (r == a.n_el - 1 && alive && !(abs_le_one(p.x) && abs_le_one(p.y))) {
      alive = false;
      code = -3;
      lturn = a.turn;
      lelem = a.n_el - 1;
    }
    double* o = a.out + (int64_t)r * 8 * n + i;
    o[0] = p.x; o[n] = p.px; o[2 * n] = p.y; o[3 * n] = p.py;
    o[4 * n] = p.zeta; o[5 * n] = p.ptau; o[6 * n] = p.delta; o[7 * n] = (double)code;
  }
  a.x[i] = p.x; a.px[i] = p.px; a.y[i] = p.y; a.py[i] = p.py; a.zeta[i] = p.zeta;
  a.delta[i] = p.delta; a.ptau[i] = p.ptau; a.rpp[i] = p.rpp; a.rvv[i] = p.rvv;
  if (alive) {  // survivors: the turn count advances, as in the tracking kernel
    lturn = a.turn + 1;
    lelem = 0;
  }
  a.state[i] = code;
  a.at_turn[i] = lturn;
  a.at_element[i] = lelem;
}

int launch_monitor(const MonitorArgs& a, int rad, void* stream) {
  if (a.n == 0 || a.n_el == 0) return 0;
  const int block = 128;
  const int grid = (int)((a.n + block - 1) / block);
  cudaStream_t s = (cudaStream_t)stream;
  if (rad == XT_RAD_MEAN) monitor_kernel<XT_RAD_MEAN><<<grid, block, 0, s>>>(a);
  else if (rad == XT_RAD_QUANTUM) monitor_kernel<XT_RAD_QUANTUM><<<grid, block, 0, s>>>(a);
  else monitor_kernel<XT_RAD_OFF><<<grid, block, 0, s>>>(a);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Order-preserving compaction of the alive particles (state == 1).
static const int CB = 1024;

__global__ void __launch_bounds__(CB) count_alive_kernel(const int32_t* __restrict__ state, int64_t n,
                                                         int32_t* __restrict__ block_counts) {
  const int64_t i = (int64_t)blockIdx.x * CB + threadIdx.x;
  const int v = (i < n) ? (state[i] == 1) : 0;
  const int c = __syncthreads_count(v);
  if (threadIdx.x == 0) block_counts[blockIdx.x] = c;
}

// Exclusive prefix sum of v over the block; *tot (shared) receives the total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* tot) {
  __shared__ int warp_sums[CB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int x = (lane < nw) ? warp_sums[lane] : 0;
    int ix = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL_MASK, ix, o);
      if (lane >= o) ix += t;
    }
    if (lane < nw) warp_sums[lane] = ix - x;
    if (lane == 31) *tot = ix;
  }
  __syncthreads();
  return warp_sums[w] + incl - v;
}

__global__ void __launch_bounds__(CB) scatter_alive_kernel(const int32_t* __restrict__ state, int64_t n,
                                                           const int32_t* __restrict__ block_counts,
                                                           int32_t* __restrict__ idx,
                                                           int32_t* __restrict__ n_alive,
                                                           int32_t* __restrict__ tile_counter) {
  __shared__ int red[CB / 32];
  __shared__ int total;
  const int b = blockIdx.x;
  // offset of this block: sum of the counts of the preceding blocks
  int s = 0;
  for (int j = threadIdx.x; j < b; j += CB) s += block_counts[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(FULL_MASK, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  int off = 0;
  for (int w = 0; w < CB / 32; w++) off += red[w];
  __syncthreads();
  const int64_t i = (int64_t)b * CB + threadIdx.x;
  const int v = (i < n) ? (state[i] == 1) : 0;
  const int pos = block_exclusive_scan(v, &total);
  if (v) idx[off + pos] = (int32_t)i;
  if (threadIdx.x == 0) {
    if (b == (int)gridDim.x - 1) *n_alive = off + total;
    if (b == 0) *tile_counter = 0;
  }
}

// Batched compaction: grid (blocks, seeds).
__global__ void __launch_bounds__(CB) count_alive_batched_kernel(const SeedDev* __restrict__ seeds,
                                                                 int32_t* __restrict__ counts,
                                                                 int32_t blocks_per_seed) {
  const int s = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * CB + threadIdx.x;
  const int64_t n = seeds[s].n;
  const int v = (i < n) ? (seeds[s].state[i] == 1) : 0;
  const int c = __syncthreads_count(v);
  if (threadIdx.x == 0) counts[(int64_t)s * blocks_per_seed + blockIdx.x] = c;
}

__global__ void __launch_bounds__(CB) scatter_alive_batched_kernel(const SeedDev* __restrict__ seeds,
                                                                   const int32_t* __restrict__ counts,
                                                                   int32_t blocks_per_seed,
                                                                   const int64_t* __restrict__ idx_base,
                                                                   int32_t* __restrict__ idx,
                                                                   int32_t* __restrict__ n_alive) {
  __shared__ int red[CB / 32];
  __shared__ int total;
  const int s = blockIdx.y, b = blockIdx.x;
  const int64_t n = seeds[s].n;
  const int nb = (int)((n + CB - 1) / CB);
  if (b >= nb) return;  // whole block exits together
  const int32_t* cnt = counts + (int64_t)s * blocks_per_seed;
  int sum = 0;
  for (int j = threadIdx.x; j < b; j += CB) sum += cnt[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(FULL_MASK, sum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  int off = 0;
  for (int w = 0; w < CB / 32; w++) off += red[w];
  __syncthreads();
  const int64_t i = (int64_t)b * CB + threadIdx.x;
  const int v = (i < n) ? (seeds[s].state[i] == 1) : 0;
  const int pos = block_exclusive_scan(v, &total);
  if (v) idx[idx_base[s] + off + pos] = (int32_t)i;
  if (threadIdx.x == 0 && b == nb - 1) n_alive[s] = off + total;
}

// tile_prefix over the seeds in processing order; also zeroes the work counter.
__global__ void tile_prefix_kernel(const int32_t* __restrict__ n_alive, const int32_t* __restrict__ order,
                                   int32_t n_seeds, int64_t* __restrict__ prefix,
                                   int32_t* __restrict__ tile_counter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t acc = 0;
    prefix[0] = 0;
    for (int j = 0; j < n_seeds; j++) {
      acc += (n_alive[order[j]] + 31) / 32;
      prefix[j + 1] = acc;
    }
    *tile_counter = 0;
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// Dynamic shared memory of a tracking block: the warps' mbarriers, two
// lattice-chunk buffers per warp, and with quantum radiation (kind 2 or 5)
// XT_PHOTON_CAP doubles per warp for the photons it samples together.
size_t track_smem_bytes(int block, int chunk_bytes, int kind) {
  const int nw = block / 32;
  const size_t photons = (kind % 3 == XT_RAD_QUANTUM) ? (size_t)nw * XT_PHOTON_CAP * sizeof(double) : 0;
  return (size_t)((nw * 16 + 127) & ~127) + (size_t)nw * 2 * (size_t)chunk_bytes + photons;
}

template <int KIND>
static int set_smem_attr(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(track_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaFuncSetAttribute(track_batched_kernel<KIND>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// kind = radiation mode (0..2) + 3 for tables with thick rows
static int smem_attr(int kind, size_t smem) {
  switch (kind) {
    case 0: return set_smem_attr<0>(smem);
    case 1: return set_smem_attr<1>(smem);
    case 2: return set_smem_attr<2>(smem);
    case 3: return set_smem_attr<3>(smem);
    case 4: return set_smem_attr<4>(smem);
    default: return set_smem_attr<5>(smem);
  }
}

int launch_track(const TrackArgs& a, int kind, int block, int grid, size_t smem, void* stream) {
  int e = smem_attr(kind, smem);
  if (e) return e;
  cudaStream_t s = (cudaStream_t)stream;
  switch (kind) {
    case 0: track_kernel<0><<<grid, block, smem, s>>>(a); break;
    case 1: track_kernel<1><<<grid, block, smem, s>>>(a); break;
    case 2: track_kernel<2><<<grid, block, smem, s>>>(a); break;
    case 3: track_kernel<3><<<grid, block, smem, s>>>(a); break;
    case 4: track_kernel<4><<<grid, block, smem, s>>>(a); break;
    default: track_kernel<5><<<grid, block, smem, s>>>(a); break;
  }
  return (int)cudaGetLastError();
}

int launch_track_batched(const BatchArgs& a, int kind, int block, int grid, size_t smem, void* stream) {
  int e = smem_attr(kind, smem);
  if (e) return e;
  cudaStream_t s = (cudaStream_t)stream;
  switch (kind) {
    case 0: track_batched_kernel<0><<<grid, block, smem, s>>>(a); break;
    case 1: track_batched_kernel<1><<<grid, block, smem, s>>>(a); break;
    case 2: track_batched_kernel<2><<<grid, block, smem, s>>>(a); break;
    case 3: track_batched_kernel<3><<<grid, block, smem, s>>>(a); break;
    case 4: track_batched_kernel<4><<<grid, block, smem, s>>>(a); break;
    default: track_batched_kernel<5><<<grid, block, smem, s>>>(a); break;
  }
  return (int)cudaGetLastError();
}

template <int KIND>
static int occ(int* bps, int block, size_t smem, bool batched) {
  if (batched) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, track_batched_kernel<KIND>, block, smem);
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, track_kernel<KIND>, block, smem);
}

static int occupancy(int kind, int block, size_t smem, int* bps, bool batched) {
  int e = smem_attr(kind, smem);
  if (e) return e;
  switch (kind) {
    case 0: return occ<0>(bps, block, smem, batched);
    case 1: return occ<1>(bps, block, smem, batched);
    case 2: return occ<2>(bps, block, smem, batched);
    case 3: return occ<3>(bps, block, smem, batched);
    case 4: return occ<4>(bps, block, smem, batched);
    default: return occ<5>(bps, block, smem, batched);
  }
}

int track_occupancy(int kind, int block, size_t smem, int* bps) { return occupancy(kind, block, smem, bps, false); }

int batched_occupancy(int kind, int block, size_t smem, int* bps) { return occupancy(kind, block, smem, bps, true); }

int launch_compact(const int32_t* state, int64_t n, int32_t* block_counts, int32_t* idx,
                   int32_t* n_alive, int32_t* tile_counter, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0) {
    cudaError_t e = cudaMemsetAsync(n_alive, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaMemsetAsync(tile_counter, 0, sizeof(int32_t), s);
  }
  const int nb = (int)((n + CB - 1) / CB);
  count_alive_kernel<<<nb, CB, 0, s>>>(state, n, block_counts);
  scatter_alive_kernel<<<nb, CB, 0, s>>>(state, n, block_counts, idx, n_alive, tile_counter);
  return (int)cudaGetLastError();
}

int launch_compact_batched(const SeedDev* seeds_dev, int32_t n_seeds, const int64_t* idx_base_dev,
                           int32_t* idx, int32_t* n_alive, int32_t* counts, int64_t max_n, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int bps = (int)((max_n + CB - 1) / CB);
  dim3 grid(bps, n_seeds);
  count_alive_batched_kernel<<<grid, CB, 0, s>>>(seeds_dev, counts, bps);
  scatter_alive_batched_kernel<<<grid, CB, 0, s>>>(seeds_dev, counts, bps, idx_base_dev, idx, n_alive);
  return (int)cudaGetLastError();
}

int launch_tile_prefix(const int32_t* n_alive, const int32_t* order, int32_t n_seeds, int64_t* prefix,
                       int32_t* tile_counter, void* stream) {
  tile_prefix_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(n_alive, order, n_seeds, prefix, tile_counter);
  return (int)cudaGetLastError();
}

__global__ void set_int_kernel(int32_t* dst, int32_t v) { *dst = v; }

// FP64 throughput probe: 16 independent fma chains per thread.
// FP64 throughput probe: CH independent fma chains per thread, all operands
// in registers.  MODE 0: a_j = a_j * m + c with m, c shared by the chains;
// MODE 1: a_j = b_j * c_j + a_j with per-chain b_j, c_j (three distinct
// register pairs per instruction).  The values stay finite and the chains
// cannot be merged, so the kernel issues exactly CH fmas per iteration.
template <int CH, int MODE>
__global__ void __launch_bounds__(128) fp64_probe_kernel(double* out, int iters) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  double a[CH], b[CH], c[CH];
#pragma unroll
  for (int j = 0; j < CH; j++) {
    a[j] = 1.0 + 1e-9 * (gid + j);
    b[j] = 1e-5 * (1.0 + 1e-3 * j + 1e-12 * gid);
    c[j] = 1e-5 * (1.0 - 1e-3 * j);
  }
  const double m = 0.9999999 + 1e-17 * (threadIdx.x & 7), cc = 1e-7 * (1.0 + 1e-9 * (threadIdx.x & 3));
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < CH; j++) a[j] = (MODE == 0) ? fma(a[j], m, cc) : fma(b[j], c[j], a[j]);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < CH; j++) s += a[j];
  out[gid] = s;
}

// variant: 0 = 8 chains shared operands, 1 = 16 chains shared operands,
// 2 = 8 chains per-chain operands, 3 = 16 chains per-chain operands.
// Returns the chains per thread through *chains.
int launch_fp64_probe(double* out, int grid, int block, int iters, int variant, int* chains, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  switch (variant) {
    case 0: fp64_probe_kernel<8, 0><<<grid, block, 0, s>>>(out, iters); *chains = 8; break;
    case 1: fp64_probe_kernel<16, 0><<<grid, block, 0, s>>>(out, iters); *chains = 16; break;
    case 2: fp64_probe_kernel<8, 1><<<grid, block, 0, s>>>(out, iters); *chains = 8; break;
    default: fp64_probe_kernel<16, 1><<<grid, block, 0, s>>>(out, iters); *chains = 16; break;
  }
  return (int)cudaGetLastError();
}

int launch_refine(const RefineArgs& a, void* stream) {
  if (a.n <= 0) return 0;
  refine_kernel<<<(unsigned)((a.n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int upload_special_table(const double* tab) {
  return (int)cudaMemcpyToSymbol(c_special, tab, XT_SPECIAL_N * sizeof(double));
}

int launch_set_int(int32_t* dst, int32_t value, void* stream) {
  set_int_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(dst, value);
  return (int)cudaGetLastError();
}

int device_smem_optin(int* bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceGetAttribute(bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
}

int device_sm_count(int* n) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev);
}

}  // namespace xt
