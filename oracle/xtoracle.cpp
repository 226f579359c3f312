// Oracle tracker: plain, slow, single-threaded FP64 CPU implementation of the
// element-by-element symplectic tracking path of the Xsuite paper (Iadarola et
// al., "Xsuite: an integrated beam physics simulation framework").
//
// TEST INFRASTRUCTURE ONLY.  This file is the independent reference against
// which the CUDA tracker is checked.  Only the test suite, the smoke check and
// the CPU-baseline leg of the benchmark may load it.  It shares no code,
// header, table or constant generator with the CUDA library.
//
// The paper prints no formulas; it states that a beam line is a sequence of
// element objects tracked turn after turn with thin-lens integration
// (section "Lattice modelling and single particle tracking"), that aperture
// elements stop tracking of particles found outside ("Particle-matter
// interaction and collimation studies"), and that synchrotron radiation has a
// "mean" and a "quantum" model for thin elements ("Synchrotron radiation models
// and compensation").  The maps below are the textbook Hamiltonian maps with
// MAD-X sign conventions, each written out from its definition with IEEE
// square roots and divisions and the C library's sin, cos, exp, expm1 and
// asin.  Three places rewrite a difference of nearly equal numbers into an
// algebraically equal form without the cancellation, because the plain
// difference would lose more digits than the comparison with the GPU allows:
//   - the energy update, delta = u / (sqrt(1+u) + 1), u = (1+delta)^2 - 1;
//   - 1 - ep/pz (drift) and 1 - 1/rvv (thick elements), from
//     (1+delta)^2 - (1 + beta0 ptau)^2 = ptau (2/beta0 + ptau) / gamma0^2;
//   - the thin dipole of the curved frame, whose field knl0 and frame term
//     hxl (1+delta) are both about 1e-3 and cancel on the design orbit: the
//     kick is (hxl - knl0) + hxl delta minus the field of the orders >= 1.
// Small-argument evaluations of entire functions use their Taylor series
// where the closed form cancels (1 - cos a, a - sin a, asin(u)/u).
// Build with -O2 -ffp-contract=off (no implicit contraction).
//
// Coordinates: x, px=Px/P0, y, py, zeta=s-beta0*c*t, delta=(P-P0)/P0,
// ptau=(E-E0)/(P0 c), rpp=1/(1+delta), rvv=beta/beta0.
//
// The scalar type is a template parameter so the same map code yields values
// (double) and exact first derivatives (Dual, forward-mode differentiation)
// for the one-turn Jacobian, the closed orbit and the optics pins.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace xo {

// ---------------------------------------------------------------------------
// Physical constants (CODATA 2018).
static const double C_LIGHT = 299792458.0;          // m/s
static const double M_ELECTRON = 0.51099895000e6;   // eV
static const double R_ELECTRON = 2.8179403262e-15;  // m
static const double ALPHA_FS = 7.2973525693e-3;
static const double HBAR_C = 197.3269804e-9;        // eV m
static const double PI = 3.14159265358979323846;

// Element descriptor: the flat lattice-table row (type, order, 48 params).
struct Element {
  int32_t type;
  int32_t order;
  double p[48];
};
enum {
  T_MARKER = 0, T_DRIFT = 1, T_MULTIPOLE = 2, T_CAVITY = 3,
  T_DIPEDGE = 4, T_LINEARMAP = 5, T_APERTURE = 6, T_XYSHIFT = 7, T_SROTATION = 8,
  T_APERTURE_RECT = 9, T_APERTURE_ELLIPSE = 10, T_BEAMBEAM4D = 11, T_QUAD = 12,
  T_BEND = 13, T_SPACECHARGE = 14
};
struct Reference { double mass0, q0, p0c; };

// ---------------------------------------------------------------------------
// Dual number with 6 infinitesimal directions (forward-mode derivative).
struct Dual {
  double v;
  double d[6];
};
static inline Dual mkd(double v) { Dual r; r.v = v; for (int i = 0; i < 6; i++) r.d[i] = 0; return r; }
static inline Dual operator+(const Dual& a, const Dual& b) { Dual r; r.v = a.v + b.v; for (int i = 0; i < 6; i++) r.d[i] = a.d[i] + b.d[i]; return r; }
static inline Dual operator-(const Dual& a, const Dual& b) { Dual r; r.v = a.v - b.v; for (int i = 0; i < 6; i++) r.d[i] = a.d[i] - b.d[i]; return r; }
static inline Dual operator-(const Dual& a) { Dual r; r.v = -a.v; for (int i = 0; i < 6; i++) r.d[i] = -a.d[i]; return r; }
static inline Dual operator*(const Dual& a, const Dual& b) { Dual r; r.v = a.v * b.v; for (int i = 0; i < 6; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
static inline Dual operator/(const Dual& a, const Dual& b) { Dual r; r.v = a.v / b.v; for (int i = 0; i < 6; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v; return r; }
static inline Dual operator+(const Dual& a, double b) { Dual r = a; r.v = a.v + b; return r; }
static inline Dual operator+(double a, const Dual& b) { Dual r = b; r.v = a + b.v; return r; }
static inline Dual operator-(const Dual& a, double b) { Dual r = a; r.v = a.v - b; return r; }
static inline Dual operator-(double a, const Dual& b) { Dual r; r.v = a - b.v; for (int i = 0; i < 6; i++) r.d[i] = -b.d[i]; return r; }
static inline Dual operator*(const Dual& a, double b) { Dual r; r.v = a.v * b; for (int i = 0; i < 6; i++) r.d[i] = a.d[i] * b; return r; }
static inline Dual operator*(double a, const Dual& b) { Dual r; r.v = a * b.v; for (int i = 0; i < 6; i++) r.d[i] = a * b.d[i]; return r; }
static inline Dual operator/(const Dual& a, double b) { Dual r; r.v = a.v / b; for (int i = 0; i < 6; i++) r.d[i] = a.d[i] / b; return r; }
static inline Dual operator/(double a, const Dual& b) { Dual r; r.v = a / b.v; for (int i = 0; i < 6; i++) r.d[i] = -r.v * b.d[i] / b.v; return r; }

static inline double val(double a) { return a; }
static inline double val(const Dual& a) { return a.v; }

// Elementary functions: the C library for values, the chain rule for duals.
static inline double SQRT(double a) { return std::sqrt(a); }
static inline double SIN(double a) { return std::sin(a); }
static inline double COS(double a) { return std::cos(a); }
static inline double EXP(double a) { return std::exp(a); }
static inline double ASIN(double a) { return std::asin(a); }
static inline Dual chain(double v, double dv, const Dual& a) {
  Dual r; r.v = v; for (int i = 0; i < 6; i++) r.d[i] = dv * a.d[i]; return r;
}
static inline Dual SQRT(const Dual& a) { const double s = std::sqrt(a.v); return chain(s, 0.5 / s, a); }
static inline Dual SIN(const Dual& a) { return chain(std::sin(a.v), std::cos(a.v), a); }
static inline Dual COS(const Dual& a) { return chain(std::cos(a.v), -std::sin(a.v), a); }
static inline Dual EXP(const Dual& a) { const double e = std::exp(a.v); return chain(e, e, a); }
static inline Dual ASIN(const Dual& a) { return chain(std::asin(a.v), 1.0 / std::sqrt(1.0 - a.v * a.v), a); }

template <class T> static inline T mkv(double v);
template <> inline double mkv<double>(double v) { return v; }
template <> inline Dual mkv<Dual>(double v) { return mkd(v); }

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based RNG.
// Counter = (particle id, turn, element index, call index); key = (seed, 0).
// This is the one generator both implementations write from its published
// definition; the method's random numbers are its output words.
static inline void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  __uint128_t p = (__uint128_t)a * (__uint128_t)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}
void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
    mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}
// 53-bit uniform in [0, 1) from a 64-bit word: (w >> 11) / 2^53.
static inline double u01(uint64_t w) { return (double)(w >> 11) / 9007199254740992.0; }

// Stream of uniforms for one (particle, turn, element): four per Philox call.
struct Uniforms {
  uint64_t ctr[4], key[2], buf[4];
  int pos;
  Uniforms(uint64_t seed, uint64_t pid, uint64_t turn, uint64_t elem) {
    ctr[0] = pid; ctr[1] = turn; ctr[2] = elem; ctr[3] = 0;
    key[0] = seed; key[1] = 0; pos = 4;
  }
  double next() {
    if (pos == 4) { philox4x64_10(ctr, key, buf); ctr[3] += 1; pos = 0; }
    return u01(buf[pos++]);
  }
};

// ---------------------------------------------------------------------------
// Photon spectrum for the quantum radiation model.  The number of photons per
// unit energy fraction xi = u/u_c is proportional to G(xi) = int_xi^inf
// K_{5/3}(t) dt, normalised by int_0^inf G = 5*pi/3.  Using the integral
// representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt and exchanging
// the order of integration, the survival function is
//   S(xi) = int_xi^inf G(s) ds = int_0^inf exp(-xi cosh t) cosh(5t/3)/cosh^2 t dt,
// and the cumulative distribution is F(xi) = 1 - S(xi)/(5 pi/3).  S is
// evaluated by the trapezoidal rule in t (the integrand is even and analytic in
// the strip |Im t| < pi/2, so the rule converges geometrically).  The sampler
// (a reading: the paper cites Burkhardt's method, whose text is absent) is the
// inverse of the piecewise-linear interpolant of F through 2048 knots
// log-spaced on [1e-7, 40], with the small-xi asymptote F ~ xi^(1/3) below the
// first knot and a clamp above the last.
static const int SPEC_K = 2048;
static const double SPEC_XI_MIN = 1e-7, SPEC_XI_MAX = 40.0;
struct Spectrum {
  double xi[SPEC_K], F[SPEC_K];
  Spectrum() {
    const double norm = 5.0 * PI / 3.0, h = 0.05;
    for (int i = 0; i < SPEC_K; i++) {
      double e = (double)i / (double)(SPEC_K - 1);
      double x = SPEC_XI_MIN * std::pow(SPEC_XI_MAX / SPEC_XI_MIN, e);
      double s = 0.0;
      for (int j = 0;; j++) {
        double t = j * h;
        double ch = std::cosh(t);
        double g = std::exp(-x * ch) * std::cosh(5.0 * t / 3.0) / (ch * ch);
        s += (j == 0 ? 0.5 : 1.0) * g;
        if (x * ch > 60.0 && j > 10) break;
      }
      xi[i] = x;
      F[i] = 1.0 - (h * s) / norm;
    }
  }
  // Inverse of the interpolated CDF at u in [0, 1): the knot interval
  // lo = max{i : F[i] <= u} is found by binary search.
  double sample(double u) const {
    if (u < F[0]) { double q = u / F[0]; return xi[0] * q * q * q; }
    if (u >= F[SPEC_K - 1]) return xi[SPEC_K - 1];
    const int lo = (int)(std::upper_bound(F, F + SPEC_K, u) - F) - 1;
    const int hi = lo + 1;
    const double w = (u - F[lo]) / (F[hi] - F[lo]);
    return xi[lo] + w * (xi[hi] - xi[lo]);
  }
};
static const Spectrum& spectrum() { static Spectrum s; return s; }

// ---------------------------------------------------------------------------
// Reference-derived constants.
struct RefConst {
  double m0, q0, p0c, E0, beta0, gamma0, bg0, ib0, twoib0, ig02;
  double crad;   // (2/3) r_c m0 / p0c   [m]
  double kq;     // (5 / (2 sqrt 3)) alpha q0^2  (mean photon count per gamma*h*L)
  double uc15;   // 1.5 hbar c  [eV m]
};
static RefConst ref_const(const Reference& r) {
  RefConst c;
  c.m0 = r.mass0; c.q0 = r.q0; c.p0c = r.p0c;
  c.E0 = std::sqrt(r.p0c * r.p0c + r.mass0 * r.mass0);
  c.beta0 = r.p0c / c.E0;
  c.gamma0 = c.E0 / r.mass0;
  c.bg0 = r.p0c / r.mass0;
  c.ib0 = c.E0 / r.p0c;
  c.twoib0 = 2.0 * c.ib0;
  c.ig02 = (r.mass0 / c.E0) * (r.mass0 / c.E0);  // 1/gamma0^2
  const double rc = r.q0 * r.q0 * R_ELECTRON * M_ELECTRON / r.mass0;
  c.crad = 2.0 * rc * r.mass0 / (3.0 * r.p0c);
  c.kq = 5.0 * ALPHA_FS * r.q0 * r.q0 / (2.0 * std::sqrt(3.0));
  c.uc15 = 1.5 * HBAR_C;
  return c;
}

// ---------------------------------------------------------------------------
// Field of a bi-Gaussian line charge (section "Beam-beam interactions"; the
// frozen model of section "Space charge").  For a unit line charge with rms
// sizes sigma_x, sigma_y, f = E 2 pi eps0 / lambda is the single integral
//   f_x = x int_0^inf exp(-x^2/(2sx^2+q) - y^2/(2sy^2+q)) / ((2sx^2+q)^(3/2) (2sy^2+q)^(1/2)) dq,
// f_y the same with the exponents 3/2 and 1/2 exchanged.  With c = min(2sx^2,
// 2sy^2) and q = c (1 - t)/t it is an integral over t in (0, 1] of a bounded
// analytic function,
//   f_x = x c int_0^1 exp(-t (x^2/Ax + y^2/Ay)) / (Ax^(3/2) Ay^(1/2)) dt,
//   Ax = c + (2sx^2 - c) t >= c,  Ay = c + (2sy^2 - c) t >= c,
// whose mass sits at t ~ 1/R for a particle at R = (x^2 + y^2)/c >> 1.  With
// t = exp(-w) the integrand is smooth on the scale of one unit of w (the
// Gaussian's own decay near w = ln R, the change of Ax or Ay from c to
// 2s^2 near w = ln(2s^2/c)), and the integral over w in [0, W],
// W = 40 + ln max(1, R) (the rest is below e^-40 of it), is taken by the
// 16-point Gauss-Legendre rule on unit intervals.  A round beam (sx == sy) has the closed form
// f = (x, y)(1 - exp(-r^2/(2 s^2)))/r^2.

// Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1]: Newton's
// method on P_n from the three-term recurrence (n + 1) P_(n+1) = (2n + 1) x P_n - n P_(n-1).
struct GaussLegendre {
  static const int N = 16;
  double x[N], w[N];
  GaussLegendre() {
    for (int i = 0; i < N; i++) {
      double z = std::cos(PI * (i + 0.75) / (N + 0.5));
      for (int it = 0; it < 100; it++) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= N; k++) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / (double)k;
          p0 = p1;
          p1 = p2;
        }
        const double dp = N * (z * p1 - p0) / (z * z - 1.0);  // P_n'
        const double dz = p1 / dp;
        z = z - dz;
        if (std::fabs(dz) < 1e-17 || it == 99) {
          double q0 = 1.0, q1 = z;
          for (int k = 2; k <= N; k++) {
            const double q2 = ((2.0 * k - 1.0) * z * q1 - (k - 1.0) * q0) / (double)k;
            q0 = q1;
            q1 = q2;
          }
          const double d = N * (z * q1 - q0) / (z * z - 1.0);
          x[i] = z;
          w[i] = 2.0 / ((1.0 - z * z) * d * d);
          break;
        }
      }
    }
  }
};
static const GaussLegendre& gauss_legendre() { static GaussLegendre g; return g; }

// f = (f_x, f_y) at (x, y) about the charge's centre.
static void gauss_field(double x, double y, double sx, double sy, double* fx, double* fy) {
  const double x2 = x * x, y2 = y * y;
  if (sx == sy) {
    const double r2 = x2 + y2;
    const double s2 = 2.0 * sx * sx;
    const double g = (r2 == 0.0) ? 1.0 / s2 : -std::expm1(-r2 / s2) / r2;
    *fx = x * g;
    *fy = y * g;
    return;
  }
  const double a = 2.0 * sx * sx, b = 2.0 * sy * sy, c = std::min(a, b);
  const double R = (x2 + y2) / c;
  const int nw = (int)std::ceil(40.0 + std::log(std::max(1.0, R)));
  const GaussLegendre& g = gauss_legendre();
  double ix = 0.0, iy = 0.0;
  for (int k = 0; k < nw; k++) {
    const double mid = k + 0.5;
    for (int i = 0; i < GaussLegendre::N; i++) {
      const double w = mid + 0.5 * g.x[i];
      const double t = std::exp(-w);
      const double Ax = c + (a - c) * t, Ay = c + (b - c) * t;
      const double e = std::exp(-t * (x2 / Ax + y2 / Ay));
      const double q = g.w[i] * 0.5 * t * e / (std::sqrt(Ax) * std::sqrt(Ay));
      ix += q / Ax;
      iy += q / Ay;
    }
  }
  *fx = x * (c * ix);
  *fy = y * (c * iy);
}

// ---------------------------------------------------------------------------
// Particle state.
template <class T>
struct Part {
  T x, px, y, py, zeta, delta, ptau, rpp, rvv;
  int32_t state, at_turn, at_element;
  int64_t id;
};

// (1+delta)^2 - (1 + beta0 ptau)^2 = ptau (2/beta0 + ptau) / gamma0^2, the
// difference of the squared relative momentum and the squared energy factor
// 1 + beta0 ptau = (1+delta)/rvv, written without cancellation.
template <class T>
static inline T dsq_mom_energy(const Part<T>& p, const RefConst& rc) {
  return (p.ptau * (rc.twoib0 + p.ptau)) * rc.ig02;
}

// Energy update from a new ptau: (1+delta)^2 = 1 + 2 ptau/beta0 + ptau^2, so
// delta = sqrt(1+u) - 1 with u = ptau (ptau + 2/beta0), evaluated as
// u / (sqrt(1+u) + 1); then rpp = 1/(1+delta) and rvv = (1+delta)/(1 + beta0 ptau).
template <class T>
static inline void energy_update(Part<T>& p, const RefConst& rc) {
  const T u = p.ptau * (p.ptau + rc.twoib0);
  p.delta = u / (SQRT(1.0 + u) + 1.0);
  p.rpp = 1.0 / (1.0 + p.delta);
  p.rvv = (1.0 + p.delta) / (1.0 + rc.beta0 * p.ptau);
}

template <class T>
static inline void mark_lost(Part<T>& p, int code, int turn, int elem) {
  p.state = code; p.at_turn = turn; p.at_element = elem;
}

// Exact drift of length L (thin-lens integration: drifts between kicks).
//   pz = sqrt((1+delta)^2 - px^2 - py^2),  x += px L/pz,  y += py L/pz,
//   zeta += L - (1+delta)/rvv * L/pz  (path length L(1+delta)/pz at speed beta).
// With ep = (1+delta)/rvv = 1 + beta0 ptau the zeta step is L (pz - ep)/pz
// = L (pz^2 - ep^2) / (pz (pz + ep)), and pz^2 - ep^2 =
// ptau (2/beta0 + ptau)/gamma0^2 - px^2 - py^2.  A particle with pz^2 <= 0
// (or not finite) is lost (code -2) with its coordinates unchanged.
template <class T>
static inline void drift(Part<T>& p, double L, const RefConst& rc, int turn, int elem) {
  const T opd = 1.0 + p.delta;
  const T pz2 = opd * opd - p.px * p.px - p.py * p.py;
  if (!(val(pz2) > 0.0 && val(pz2) < INFINITY)) { mark_lost(p, -2, turn, elem); return; }
  const T pz = SQRT(pz2);
  const T lpz = L / pz;
  const T ep = 1.0 + rc.beta0 * p.ptau;
  const T num = dsq_mom_energy(p, rc) - p.px * p.px - p.py * p.py;
  p.x = p.x + p.px * lpz;
  p.y = p.y + p.py * lpz;
  p.zeta = p.zeta + L * num / (pz * (pz + ep));
}

// Energy change by radiation: ptau += dpt, then the energy update; the
// transverse momenta are scaled by (1+delta_new)/(1+delta_old) so that the
// angles px/(1+delta), py/(1+delta) are unchanged (emission along the motion).
template <class T>
static inline void apply_energy_loss(Part<T>& p, T dpt, const RefConst& rc) {
  const T opd_old = 1.0 + p.delta;
  p.ptau = p.ptau + dpt;
  energy_update(p, rc);
  const T f = (1.0 + p.delta) / opd_old;
  p.px = p.px * f;
  p.py = p.py * f;
}

// Per-element constants of a thin multipole: c_n = knl_n/n!, s_n = ksl_n/n!,
// the frame curvature hxl, the radiation length L_rad, and
// k0h = knl0 hxl / L_rad (0 when L_rad == 0).
struct MultConst {
  int N;
  double c[11], s[11];
  double hxl, k0h, lrad;
};

// Quantum model: Poisson number of photons with mean
// nbar = (5/(2 sqrt 3)) alpha q0^2 gamma h L_rad, drawn by sequential
// inversion (p_0 = e^(-nbar), p_k = p_(k-1) nbar / k, at most 200 photons),
// energies u = u_c xi with u_c = (3/2) hbar c gamma^3 h and xi from the
// spectrum sampler, one uniform each, after the Poisson uniform.
static const int KMAX_PHOTONS = 200;
static inline void quantum_kick(Part<double>& p, double br, double bi, const MultConst& m,
                                const RefConst& rc, uint64_t seed, int turn, int elem) {
  const double h = std::sqrt(br * br + bi * bi) / (m.lrad * (1.0 + p.delta));
  const double gam = rc.gamma0 + rc.bg0 * p.ptau;
  const double nbar = rc.kq * m.lrad * gam * h;
  Uniforms U(seed, (uint64_t)p.id, (uint64_t)turn, (uint64_t)elem);
  const double u0 = U.next();
  int k = 0;
  double pk = std::exp(-nbar), F = pk;
  while (u0 > F && k < KMAX_PHOTONS) { k++; pk = pk * nbar / (double)k; F = F + pk; }
  if (k == 0) return;
  const Spectrum& S = spectrum();
  double sxi = 0.0;
  for (int j = 0; j < k; j++) sxi = sxi + S.sample(U.next());
  const double uc = rc.uc15 * gam * gam * gam * h;
  apply_energy_loss(p, -(uc * sxi) / rc.p0c, rc);
}
static inline void quantum_kick(Part<Dual>&, const Dual&, const Dual&, const MultConst&,
                                const RefConst&, uint64_t, int, int) {}

// Field of the orders >= 1 of a thin multipole at z = x + i y:
// sum_{n>=1} (c_n + i s_n) z^n by Horner's rule from the top order.
template <class T>
static inline void multipole_field(const Part<T>& p, const MultConst& m, T* fr, T* fi) {
  *fr = mkv<T>(0.0);
  *fi = mkv<T>(0.0);
  if (m.N < 1) return;
  T ar = mkv<T>(m.c[m.N]), ai = mkv<T>(m.s[m.N]);
  for (int n = m.N - 1; n >= 1; n--) {
    const T nr = ar * p.x - ai * p.y + m.c[n];
    const T ni = ar * p.y + ai * p.x + m.s[n];
    ar = nr;
    ai = ni;
  }
  *fr = ar * p.x - ai * p.y;
  *fi = ar * p.y + ai * p.x;
}

// Thin multipole: b = sum_n (knl_n + i ksl_n) z^n / n!; px -= Re b, py += Im b.
// With a curvature hxl the thin dipole of the curved frame adds
// px += hxl (1+delta) - knl0 hxl x / L_rad and zeta -= hxl x / rvv.  The
// constant term -knl0 and hxl (1+delta) are added to px together, as
// (hxl - knl0) + hxl delta: each is about 1e-3 in a ring's dipole slice while
// their sum on the design orbit is 0, and px itself is about 1e-5.
// Radiation (mode 1 mean, 2 quantum) is applied once, after the kick, for
// elements with L_rad > 0, from the field kick b only.
template <class T>
static inline void multipole(Part<T>& p, const MultConst& m, int rad_mode, const RefConst& rc,
                             uint64_t seed, int turn, int elem) {
  T fr, fi;
  multipole_field(p, m, &fr, &fi);
  p.px = p.px - fr;
  p.py = p.py + fi + m.s[0];
  if (m.hxl != 0.0) {
    p.px = p.px + ((m.hxl - m.c[0]) + m.hxl * p.delta);
    p.px = p.px - m.k0h * p.x;
    p.zeta = p.zeta - m.hxl * p.x / p.rvv;
  } else {
    p.px = p.px - m.c[0];
  }
  if (rad_mode == 0 || !(m.lrad > 0.0)) return;
  const T br = fr + m.c[0], bi = fi + m.s[0];
  if (rad_mode == 1) {
    // Mean model: dE = -(2/3) r_c m0 c^2 beta^3 gamma^4 h^2 L_rad with the local
    // curvature h = |b| / ((1+delta) L_rad).
    const T h = SQRT(br * br + bi * bi) / (m.lrad * (1.0 + p.delta));
    const T gam = rc.gamma0 + rc.bg0 * p.ptau;
    const T bet = rc.beta0 * p.rvv;
    const T dpt = -(rc.crad * m.lrad) * (bet * bet * bet) * (gam * gam * gam * gam) * (h * h);
    apply_energy_loss(p, dpt, rc);
  } else {
    quantum_kick(p, br, bi, m, rc, seed, turn, elem);
  }
}

// ---------------------------------------------------------------------------
// Entire functions of z (either sign) with a = sqrt|z|: C = cos a,
// S = sin(a)/a, S2 = (1 - cos a)/z, S3 = (1 - S)/z for z > 0, and cosh a,
// sinh(a)/a, (1 - cosh a)/z, (1 - S)/z for z < 0.  For |z| < 1/2 their Taylor
// series C = sum (-z)^k/(2k)!, S = sum (-z)^k/(2k+1)!, S2 = sum (-z)^k/(2k+2)!,
// S3 = sum (-z)^k/(2k+3)! to k = 12 (truncation below 1e-28); otherwise the
// closed forms with 1 - cos a = 2 sin^2(a/2) and cosh a - 1 = 2 sinh^2(a/2).
static const std::vector<double>& inv_fact() {
  static std::vector<double> c = [] {
    std::vector<double> v(32);
    double f = 1.0;
    for (int n = 0; n < 32; n++) {
      if (n > 0) f = f * (double)n;
      v[n] = 1.0 / f;
    }
    return v;
  }();
  return c;
}
template <class T>
static inline void osc_funcs(const T& z, T* C, T* S, T* S2, T* S3) {
  if (std::fabs(val(z)) < 0.5) {
    const std::vector<double>& f = inv_fact();
    const T mz = -z;
    T c = mkv<T>(f[24]), s = mkv<T>(f[25]), s2 = mkv<T>(f[26]), s3 = mkv<T>(f[27]);
    for (int k = 11; k >= 0; k--) {
      c = c * mz + f[2 * k];
      s = s * mz + f[2 * k + 1];
      s2 = s2 * mz + f[2 * k + 2];
      s3 = s3 * mz + f[2 * k + 3];
    }
    *C = c; *S = s; *S2 = s2; *S3 = s3;
    return;
  }
  if (val(z) > 0.0) {
    const T a = SQRT(z);
    const T sh = SIN(0.5 * a);
    *C = COS(a);
    *S = SIN(a) / a;
    *S2 = 2.0 * sh * sh / z;
  } else {
    const T a = SQRT(-z);
    const T e = EXP(a), ei = EXP(-a);
    const T eh = EXP(0.5 * a), ehi = EXP(-0.5 * a);
    const T sh = 0.5 * (eh - ehi);  // sinh(a/2)
    *C = 0.5 * (e + ei);
    *S = (0.5 * (e - ei)) / a;
    *S2 = 2.0 * sh * sh / (-z);
  }
  *S3 = (1.0 - *S) / z;
}

// Thick quadrupole: the exact flow over L of the expanded Hamiltonian
// H = pzeta - (1+delta) + (px^2 + py^2) / (2 (1+delta)) + k1 (x^2 - y^2) / 2
// (section "Lattice modelling and single particle tracking" names thick
// quadrupoles).  With w^2 = |k1|/(1+delta) the focusing plane (x for k1 >= 0)
// has u = u0 cos(ws) + pu0 sin(ws)/(w (1+delta)), pu = (1+delta) u', the other
// the same with cosh and sinh; and zeta' = 1 - (1/rvv)(1 + (px^2 + py^2)/(2 (1+delta)^2)).
// Over the body, int cos^2 = (L/2)(1 + C Sa), int sin^2 = (L/2)(1 - C Sa) and
// int sin cos = w L^2 Sa^2 / 2 with C = cos(wL), Sa = sin(wL)/(wL) (the
// hyperbolic ones alike), which gives int (px^2 + py^2) ds in closed form.
// The sign of L is carried through: the map with -L is the inverse.
template <class T>
static inline void thick_quad(Part<T>& p, double k1, double L, const RefConst& rc) {
  if (L == 0.0) return;
  const T opd = 1.0 + p.delta;
  const double ak1 = std::fabs(k1);
  const T aK = ak1 / opd;  // w^2
  const T z = aK * (L * L);
  T C, Sa, Ch, Sha, u2, u3;
  osc_funcs(z, &C, &Sa, &u2, &u3);
  osc_funcs(-z, &Ch, &Sha, &u2, &u3);
  T* u = (k1 >= 0.0) ? &p.x : &p.y;
  T* pu = (k1 >= 0.0) ? &p.px : &p.py;
  T* v = (k1 >= 0.0) ? &p.y : &p.x;
  T* pv = (k1 >= 0.0) ? &p.py : &p.px;
  const T u0 = *u, pu0 = *pu, v0 = *v, pv0 = *pv;
  *u = C * u0 + (L * Sa / opd) * pu0;
  *pu = C * pu0 - (aK * L * Sa) * opd * u0;
  *v = Ch * v0 + (L * Sha / opd) * pv0;
  *pv = Ch * pv0 + (aK * L * Sha) * opd * v0;
  const T A2 = pu0 * pu0, B2 = opd * ak1 * (u0 * u0);     // pu0^2, (opd w u0)^2
  const T Ah2 = pv0 * pv0, Bh2 = opd * ak1 * (v0 * v0);
  const double hL = 0.5 * L;
  const T I = hL * (1.0 + C * Sa) * A2 + hL * (1.0 - C * Sa) * B2 - opd * aK * (L * L) * (Sa * Sa) * (pu0 * u0)
            + hL * (1.0 + Ch * Sha) * Ah2 + hL * (Ch * Sha - 1.0) * Bh2 + opd * aK * (L * L) * (Sha * Sha) * (pv0 * v0);
  // 1 - 1/rvv = ((1+delta)^2 - ep^2) / ((1+delta)((1+delta) + ep)), ep = 1 + beta0 ptau
  const T ep = 1.0 + rc.beta0 * p.ptau;
  const T one_m_irvv = dsq_mom_energy(p, rc) / (opd * (opd + ep));
  p.zeta = p.zeta + L * one_m_irvv - I / (2.0 * p.rvv * opd * opd);
}

// Dipole edge, non-linear model (section "Lattice modelling and single
// particle tracking": edge effects as full non-linear maps).  A hard edge of
// the field k0 whose face makes the angle e with the normal to the reference
// orbit.  To first order in the field gradient, Maxwell's equations attach
// B_s = y dB_y/ds and B_x = -tan(e) y dB_y/ds to it; across the edge they
// kick py -= k0 y T with T = tan(e + s atan(px/pz)) (s = +1 at the entrance,
// -1 at the exit), and the field missing from (or added to) the wedge between
// the face and the normal plane gives px += k0 tan(e) x.  The map is the
// canonical transformation of the type-2 generating function
//   x X' + y Y' + zeta Z' + (k0/2) y^2 T(Px', Py', delta) - (k0/2) tan(e) x^2:
// Py' = py - k0 y T(px, Py') is solved by fixed-point iteration until it no
// longer changes, and X', Y', Z' = (x, y, zeta) + (k0/2) y^2 dT/d(px, py, pzeta) with
//   dT/dpx = s (1+t^2)(pz^2 + px^2)/(pz D^2), dT/dpy = s (1+t^2) px py/(pz D^2),
//   dT/dpzeta = -s (1+t^2) px (1+delta)/(pz D^2 rvv), D = pz - s t px, t = tan(e),
// and the wedge kick after it at the entrance, before it at the exit.  The
// finite extent of the fringe (fint, hgap) enters as in the linear model: a
// further py += (h tan(e) - h tan(e - psi)) y, so that the linearisation at
// the origin is the linear edge.  Lost with code -2 if pz is not real.
template <class T>
static inline void edge_nonlinear(Part<T>& p, double k0, double t, double sgn, double r21, double corr,
                                  int turn, int elem) {
  if (sgn < 0.0) p.px = p.px + r21 * p.x;
  const T px = p.px, y = p.y, py = p.py;
  const T opd = 1.0 + p.delta;
  const T base = opd * opd - px * px;  // pz^2 + py^2
  if (!(val(base - py * py) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
  const T ky = k0 * y;
  T pyn = py;
  for (int k = 0; k < 60; k++) {
    const T pz2 = base - pyn * pyn;
    if (!(val(pz2) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
    const T pz = SQRT(pz2);
    const T Tv = (t * pz + sgn * px) / (pz - sgn * t * px);
    const T nxt = py - ky * Tv;
    const bool same = val(nxt) == val(pyn);
    pyn = nxt;
    if (same && k >= 3) break;
  }
  const T pz2 = base - pyn * pyn;
  if (!(val(pz2) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
  const T pz = SQRT(pz2);
  const T D = pz - sgn * t * px;
  const T c = (sgn * (1.0 + t * t)) / (pz * D * D);
  const T g = 0.5 * k0 * (y * y) * c;
  p.x = p.x + g * (pz * pz + px * px);
  p.y = p.y + g * (px * pyn);
  p.zeta = p.zeta - g * px * opd / p.rvv;
  p.py = pyn + corr * p.y;
  if (sgn > 0.0) p.px = p.px + r21 * p.x;
}

// Change of reference plane (exact wedge geometry of a bend's inclined pole
// face; section "Lattice modelling and single particle tracking": bends and
// their edge effects).  The new plane is the old one rotated by the angle a
// (cos a = ca, sin a = sa) about the vertical axis through the reference
// point; between the two planes the particle moves in the uniform vertical
// field k0 (k0 = 0: a straight line).  In the rotated axes the particle starts
// at X = x ca, Z = -x sa with momenta px2 = px ca + pz sa, pzr = pz ca - px sa.
// Circular motion keeps pX + k0 Z and pZ - k0 X, so on the new plane (Z = 0)
//   px' = px2 - k0 x sa,
//   x'  = x ca + (pz' - pzr)/k0 = x ca + x sa (px2 + px')/(pz' + pzr),
// the second form from pz'^2 - pzr^2 = px2^2 - px'^2.  The direction turns by
// dpsi with sin(dpsi) = (px2 pz' - pzr px')/p_h^2 = k0 G/p_h^2,
// G = x sa (pzr + px2 (px2 + px')/(pz' + pzr)), and the horizontal path is
// p_h dpsi/k0 = p_h (G/p_h^2) asin(v)/v, v = k0 G/p_h^2 (for k0 = 0 the
// straight path to the plane).  y and zeta follow the path as in a drift:
// y += py lr, zeta -= (1+delta) lr/rvv, lr = path/p_h; the plane has no
// reference length.  Lost with code -2 if pz or pz' is not real or the plane
// is not reached.
template <class T>
static inline T asin_over(const T& u);
template <class T>
static inline void plane_rotation(Part<T>& p, double k0, double ca, double sa, int turn, int elem) {
  const T opd = 1.0 + p.delta;
  const T ph2 = opd * opd - p.py * p.py;
  const T pz2 = ph2 - p.px * p.px;
  if (!(val(pz2) > 0.0 && val(pz2) < INFINITY)) { mark_lost(p, -2, turn, elem); return; }
  const T pz = SQRT(pz2);
  const T px2 = p.px * ca + pz * sa;
  const T pzr = pz * ca - p.px * sa;
  const T xs = p.x * sa;
  const T pxf = px2 - k0 * xs;
  const T pzf2 = ph2 - pxf * pxf;
  if (!(val(pzf2) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
  const T pzf = SQRT(pzf2);
  const T den = pzf + pzr;
  if (!(val(den) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
  const T q = (px2 + pxf) / den;
  const T G = xs * (pzr + px2 * q);
  const T v = k0 * G / ph2;
  if (!(std::fabs(val(v)) <= 1.0)) { mark_lost(p, -2, turn, elem); return; }
  const T lr = (G / ph2) * asin_over(v);
  p.x = p.x * ca + xs * q;
  p.px = pxf;
  p.y = p.y + p.py * lr;
  p.zeta = p.zeta - lr * opd / p.rvv;
}

// Dipole edge with the exact wedge (model 2): the non-linear edge's fringe
// taken on the pole face itself, between exact changes of plane.  At the
// entrance the particle goes in a straight line from the plane normal to the
// orbit to the face (rotated by e), receives the fringe there (the face is
// its own normal plane, so the fringe's angle is the particle's angle to it:
// t = 0), and then moves in the field k0 back to the normal plane (rotation
// by -e).  The exit runs the mirror sequence: in the field to the face, the
// fringe, a straight line to the normal plane.  To first order this is the
// linear edge: px += k0 tan(e) x, py -= k0 tan(e - psi) y.
template <class T>
static inline void edge_wedge(Part<T>& p, double k0, double ce, double se, double sgn, double corr, int turn,
                              int elem) {
  if (sgn > 0.0) {
    plane_rotation(p, 0.0, ce, se, turn, elem);
    if (p.state != 1) return;
    edge_nonlinear(p, k0, 0.0, sgn, 0.0, corr, turn, elem);
    if (p.state != 1) return;
    plane_rotation(p, k0, ce, -se, turn, elem);
  } else {
    plane_rotation(p, k0, ce, -se, turn, elem);
    if (p.state != 1) return;
    edge_nonlinear(p, k0, 0.0, sgn, 0.0, corr, turn, elem);
    if (p.state != 1) return;
    plane_rotation(p, 0.0, ce, se, turn, elem);
  }
}

// asin(u)/u for |u| <= 1: the series sum_n (2n)!/(4^n n!^2 (2n+1)) u^(2n)
// below |u| = 0.1 (to n = 12), asin(u)/u above.
template <class T>
static inline T asin_over(const T& u) {
  if (std::fabs(val(u)) >= 0.1) return ASIN(u) / u;
  const T z = u * u;
  std::vector<double> a(13);
  double tn = 1.0;
  for (int n = 0; n < 13; n++) {
    if (n > 0) tn = tn * (double)(2 * n - 1) / (double)(2 * n);
    a[n] = tn / (double)(2 * n + 1);
  }
  T s = mkv<T>(a[12]);
  for (int n = 11; n >= 0; n--) s = s * z + a[n];
  return s;
}

// Thick bend, expanded model (section "Lattice modelling and single particle
// tracking": the model for large machines and small bending angles): the
// exact flow of
//   (px^2 + py^2) / (2 (1+delta)) - h x (1+delta) + k0 (x + h x^2 / 2) + k1 (x^2 - y^2) / 2,
// the Hamiltonian in the frame of curvature h with its square root expanded
// to second order in px, py and the factor (1 + h x) kept on the leading term
// only.  x is a driven oscillator, px' = F - Kx x with F = h (1+delta) - k0
// (evaluated as (h - k0) + h delta) and Kx = k0 h + k1; y has py' = k1 y; so
// with z = K L^2 / (1+delta) and the functions of osc_funcs,
//   x = C x0 + (L S/(1+delta)) px0 + (L^2 S2/(1+delta)) F,  px = C px0 + L S (F - Kx x0),
// and zeta' = 1 - (1/rvv)(1 + h x + (px^2 + py^2)/(2 (1+delta)^2)) integrates with
//   int x = L S x0 + (L^2 S2/(1+delta)) px0 + (L^3 S3/(1+delta)) F,
//   int px^2 = (L/2)(1 + C S) px0^2 + L^2 S^2 px0 G + (L^3/2) ((1 - C S)/z) G^2,
// G = F - Kx x0, where (1 - C S)/z = (2a - sin 2a)/(2 a^3) = 4 S3(4z).
// The sign of L is carried through (-L inverts).
template <class T>
static inline void bend_expanded(Part<T>& p, double k0, double h, double L, double k1, const RefConst& rc) {
  const T opd = 1.0 + p.delta;
  const double Kx = k0 * h + k1, L2 = L * L;
  const T zx = Kx * L2 / opd;
  const T zy = (-k1) * L2 / opd;
  T C, S, S2, S3, Cy, Sy, S2y, S3y, t0, t1, t2, Q, Qy;
  osc_funcs(zx, &C, &S, &S2, &S3);
  osc_funcs(zy, &Cy, &Sy, &S2y, &S3y);
  osc_funcs(4.0 * zx, &t0, &t1, &t2, &Q);
  osc_funcs(4.0 * zy, &t0, &t1, &t2, &Qy);
  Q = 4.0 * Q;
  Qy = 4.0 * Qy;
  const T x0 = p.x, px0 = p.px, y0 = p.y, py0 = p.py;
  const T F = (h - k0) + h * p.delta;
  const T G = F - Kx * x0;
  const T Gy = k1 * y0;
  p.x = C * x0 + (L * S / opd) * px0 + (L2 * S2 / opd) * F;
  p.px = C * px0 + L * S * G;
  p.y = Cy * y0 + (L * Sy / opd) * py0;
  p.py = Cy * py0 + L * Sy * Gy;
  const T Ix = L * S * x0 + (L2 * S2 / opd) * px0 + (L2 * L * S3 / opd) * F;
  const T Ipx = 0.5 * L * (1.0 + C * S) * (px0 * px0) + L2 * (S * S) * (px0 * G) + 0.5 * L2 * L * Q * (G * G);
  const T Ipy = 0.5 * L * (1.0 + Cy * Sy) * (py0 * py0) + L2 * (Sy * Sy) * (py0 * Gy) + 0.5 * L2 * L * Qy * (Gy * Gy);
  const T ep = 1.0 + rc.beta0 * p.ptau;
  const T one_m_irvv = dsq_mom_energy(p, rc) / (opd * (opd + ep));
  p.zeta = p.zeta + L * one_m_irvv - (h * Ix + (Ipx + Ipy) / (2.0 * opd * opd)) / p.rvv;
}

// Thick bend, full model (section "Lattice modelling and single particle
// tracking": the model for small machines): the exact motion in a uniform
// vertical field k0 = B / (B rho) through a sector of curvature h and
// reference length L.  In the horizontal plane the particle runs on a circle
// of radius p_h / k0, p_h^2 = (1+delta)^2 - py^2, along which pX + k0 Z and
// pZ - k0 X are constant (X, Z laboratory coordinates about the sector's
// centre, X along the entrance x axis).  At the exit plane, turned by
// theta = h L, this gives
//   px' = B - k0 (1/h + x) sin(theta),   B = px cos + pz sin,  Q = pz cos - px sin,
//   x'  = x cos - (1 - cos)/h + (1/h + x) sin (px' + B) / (pz' + Q),
// with sin/h = L S, (1 - cos)/h = h L^2 S2 (functions of z = theta^2), so that
// h = 0 is the straight dipole.  The arc length in the horizontal plane is
// l_h = chord asin(u)/u, u = k0 chord / (2 p_h), with
// chord^2 = (x' - x)^2 + (1 + h x)(1 + h x') 2 L^2 S2; then y += py l_h / p_h
// and zeta += L - (1/rvv)(1+delta) l_h / p_h.  The sign of L is carried
// through (-L inverts).  Lost with code -2 if pz or pz' is not real or the
// particle cannot reach the exit plane.
template <class T>
static inline void bend_full(Part<T>& p, double k0, double h, double L, const RefConst& rc, int turn, int elem) {
  const double th = h * L, L2 = L * L;
  double C, S, S2, S3;
  osc_funcs(th * th, &C, &S, &S2, &S3);
  const double sn = th * S, Sh = L * S, Ch = h * L2 * S2, D2 = 2.0 * L2 * S2;
  const T opd = 1.0 + p.delta;
  const T pz2 = opd * opd - p.px * p.px - p.py * p.py;
  if (!(val(pz2) > 0.0 && val(pz2) < INFINITY)) { mark_lost(p, -2, turn, elem); return; }
  const T pz = SQRT(pz2);
  const T ph2 = opd * opd - p.py * p.py;
  const T B = p.px * C + pz * sn;
  const T Q = pz * C - p.px * sn;
  const T r0s = p.x * sn + Sh;     // (1/h + x) sin(theta)
  const T A = B - k0 * r0s;        // px at the exit plane
  const T pzf2 = ph2 - A * A;
  if (!(val(pzf2) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
  const T pzf = SQRT(pzf2);
  const T den = pzf + Q;
  if (!(val(den) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
  const T xf = p.x * C - Ch + r0s * ((A + B) / den);
  const T dxf = xf - p.x;
  const T chord = SQRT(dxf * dxf + (1.0 + h * p.x) * (1.0 + h * xf) * D2);
  const T ph = SQRT(ph2);
  const T uu = k0 * chord / (2.0 * ph);
  if (!(std::fabs(val(uu)) <= 1.0)) { mark_lost(p, -2, turn, elem); return; }
  const T lh = ((L >= 0.0) ? chord : -chord) * asin_over(uu);
  const T lr = lh / ph;
  const T ep = 1.0 + rc.beta0 * p.ptau;
  p.x = xf;
  p.px = A;
  p.y = p.y + p.py * lr;
  p.zeta = p.zeta + (L - ep * lr);
}

// Thick bend, full model with a gradient k1: no closed form, so the body is
// split into n equal slices and each slice's gradient is applied as one thin
// quadrupole kick k1 L/n at its centre, between exact uniform-field bodies
// (px -= k1 L/n x, py += k1 L/n y).  Symmetric in s, hence of second order
// in L/n and inverted by -L.  Lost bodies end the element.
template <class T>
static inline void bend_full_gradient(Part<T>& p, double k0, double h, double L, double k1, int n,
                                      const RefConst& rc, int turn, int elem) {
  const double ls = L / n, kl = k1 * ls;
  for (int i = 0; i < n; i++) {
    bend_full(p, k0, h, 0.5 * ls, rc, turn, elem);
    if (p.state != 1) return;
    p.px = p.px - kl * p.x;
    p.py = p.py + kl * p.y;
    bend_full(p, k0, h, 0.5 * ls, rc, turn, elem);
    if (p.state != 1) return;
  }
}

// Prepared element: host constants of each type.
struct Prep {
  int type;
  double L;                              // drift
  MultConst m;                           // multipole
  double krf, lagr, qv;                  // cavity
  double r21, r43;                       // dipole edge (linear model)
  int enl;                               // dipole edge: 1 = non-linear model, 2 = exact wedge
  double ece, ese;                       // exact wedge: cos(e1), sin(e1)
  double ek0, et, esg, ecorr;            // non-linear edge: field, tan(e1), +1 entrance / -1 exit,
                                         // finite-extent vertical correction
  double M[36], d[6];                    // linear map in (x,px,y,py,zeta,ptau)
  double r2;                             // aperture
  double dx, dy;                         // reference-frame shift
  double cs, sn;                         // reference-frame rotation about s
  double xmin, xmax, ymin, ymax;         // rectangular aperture
  double ia2, ib2;                       // elliptic aperture: 1/a^2, 1/b^2
  double lK, lxc, lyc, lsx, lsy;         // lens: kick strength, centre, rms sizes
  double sc_sz;                          // frozen space charge: sigma_z, 0 for a coasting beam
  double k1, Lq;                         // thick quadrupole
  double bk0, bh, bL, bk1;               // thick bend: field, curvature, length, gradient
  int bfull, bn;                         // thick bend: 1 = full model, 0 = expanded; gradient kicks (full)
};

static Prep prepare(const Element& e, const RefConst& rc) {
  Prep q;
  std::memset(&q, 0, sizeof(q));
  q.type = e.type;
  switch (e.type) {
    case T_DRIFT: q.L = e.p[0]; break;
    case T_MULTIPOLE: {
      double fact = 1.0;
      q.m.N = e.order;
      for (int n = 0; n <= 10; n++) {
        if (n > 0) fact = fact * (double)n;
        q.m.c[n] = e.p[n] / fact;
        q.m.s[n] = e.p[11 + n] / fact;
      }
      q.m.hxl = e.p[22];
      q.m.lrad = e.p[23];
      q.m.k0h = (q.m.lrad > 0.0) ? (e.p[0] * q.m.hxl) / q.m.lrad : 0.0;
      break;
    }
    case T_CAVITY: {
      const double V = e.p[0], f = e.p[1], lag = e.p[2];
      q.krf = (2.0 * PI * f) / (rc.beta0 * C_LIGHT);
      q.lagr = lag * PI / 180.0;
      q.qv = (rc.q0 * V) / rc.p0c;
      break;
    }
    case T_DIPEDGE: {
      const double h = e.p[0], e1 = e.p[1], hgap = e.p[2], fint = e.p[3];
      q.r21 = h * std::tan(e1);
      const double psi = 2.0 * h * hgap * fint * (1.0 + std::sin(e1) * std::sin(e1)) / std::cos(e1);
      q.r43 = -h * std::tan(e1 - psi);
      q.enl = (int)e.p[4];
      q.ece = std::cos(e1);
      q.ese = std::sin(e1);
      q.ek0 = h;
      q.et = std::tan(e1);
      q.esg = (e.p[5] != 0.0) ? -1.0 : 1.0;
      q.ecorr = q.r21 + q.r43;  // h tan(e1) - h tan(e1 - psi)
      break;
    }
    case T_LINEARMAP: {
      // The table gives M, d on (x,px,y,py,zeta,pzeta), pzeta = ptau/beta0;
      // in (..., ptau) row 5 is multiplied by beta0 and column 5 divided by it.
      for (int i = 0; i < 6; i++) {
        for (int j = 0; j < 6; j++) {
          double v = e.p[6 * i + j];
          if (i == 5 && j != 5) v = v * rc.beta0;
          else if (j == 5 && i != 5) v = v / rc.beta0;
          q.M[6 * i + j] = v;
        }
        q.d[i] = (i == 5) ? e.p[36 + i] * rc.beta0 : e.p[36 + i];
      }
      break;
    }
    case T_APERTURE: q.r2 = e.p[0] * e.p[0]; break;
    case T_XYSHIFT: q.dx = e.p[0]; q.dy = e.p[1]; break;
    case T_SROTATION: q.cs = std::cos(e.p[0]); q.sn = std::sin(e.p[0]); break;
    case T_APERTURE_RECT: q.xmin = e.p[0]; q.xmax = e.p[1]; q.ymin = e.p[2]; q.ymax = e.p[3]; break;
    case T_APERTURE_ELLIPSE: q.ia2 = 1.0 / (e.p[0] * e.p[0]); q.ib2 = 1.0 / (e.p[1] * e.p[1]); break;
    case T_QUAD: q.k1 = e.p[0]; q.Lq = e.p[1]; break;
    case T_BEND:
      q.bk0 = e.p[0]; q.bh = e.p[1]; q.bL = e.p[2]; q.bk1 = e.p[3]; q.bfull = (e.p[4] != 0.0);
      q.bn = (e.p[5] >= 1.0) ? (int)e.p[5] : 1;
      break;
    case T_BEAMBEAM4D: {
      // kick of a counter-moving Gaussian bunch integrated over the crossing:
      // Delta p_perp / P0 = 2 q0 q_s N_s (r_e m_e c^2 / p0 c) (1 + beta0 beta_s) /
      // (beta0 + beta_s) f(x - x_c, y - y_c)
      const double qN = e.p[0], bs = e.p[1];
      q.lK = 2.0 * rc.q0 * qN * (R_ELECTRON * M_ELECTRON) / rc.p0c * ((1.0 + rc.beta0 * bs) / (rc.beta0 + bs));
      q.lsx = e.p[2]; q.lsy = e.p[3];
      q.lxc = e.p[4]; q.lyc = e.p[5];
      break;
    }
    case T_SPACECHARGE: {
      // frozen space charge (section "Space charge", frozen model): the beam's
      // own Gaussian line charge of peak density lambda0 [1/m], electric and
      // magnetic forces cancelling to 1/gamma^2, integrated over the length L
      // the lumped element stands for:
      // Delta p_perp / P0 = 2 r_c lambda0 L / (beta0^2 gamma0^3) g(zeta) f(x - x_c, y - y_c),
      // r_c = q0^2 r_e m_e / m0, g = exp(-zeta^2 / (2 sigma_z^2)) (1 when sigma_z = 0)
      const double lam0 = e.p[0], L = e.p[4];
      const double rcl = rc.q0 * rc.q0 * R_ELECTRON * M_ELECTRON / rc.m0;
      q.lK = 2.0 * rcl * lam0 * L / (rc.beta0 * rc.beta0 * rc.gamma0 * rc.gamma0 * rc.gamma0);
      q.lsx = e.p[2]; q.lsy = e.p[3];
      q.lxc = e.p[5]; q.lyc = e.p[6];
      q.sc_sz = e.p[1];
      break;
    }
    default: break;
  }
  return q;
}

// Kick of a lens row (4D beam-beam or frozen space charge) at the particle.
static inline void lens_kick(const Prep& q, double x, double y, double zeta, double* kx, double* ky) {
  double fx, fy;
  gauss_field(x - q.lxc, y - q.lyc, q.lsx, q.lsy, &fx, &fy);
  double K = q.lK;
  if (q.type == T_SPACECHARGE && q.sc_sz > 0.0) K = K * std::exp(-(zeta * zeta) / (2.0 * q.sc_sz * q.sc_sz));
  *kx = K * fx;
  *ky = K * fy;
}

// One element.  Returns with p.state != 1 if the particle was lost here.
template <class T>
static inline void track_element(Part<T>& p, const Prep& q, int rad_mode, const RefConst& rc,
                                 uint64_t seed, int turn, int elem) {
  switch (q.type) {
    case T_DRIFT: drift(p, q.L, rc, turn, elem); break;
    case T_MULTIPOLE: multipole(p, q.m, rad_mode, rc, seed, turn, elem); break;
    case T_CAVITY: {
      // Thin RF: phase lag - k zeta, k = 2 pi f/(beta0 c); energy gain q0 V sin(phase).
      const T phi = q.lagr - q.krf * p.zeta;
      p.ptau = p.ptau + q.qv * SIN(phi);
      energy_update(p, rc);
      break;
    }
    case T_DIPEDGE:
      if (q.enl == 2) {
        edge_wedge(p, q.ek0, q.ece, q.ese, q.esg, q.ecorr, turn, elem);
      } else if (q.enl) {
        edge_nonlinear(p, q.ek0, q.et, q.esg, q.r21, q.ecorr, turn, elem);
      } else {
        p.px = p.px + q.r21 * p.x;
        p.py = p.py + q.r43 * p.y;
      }
      break;
    case T_LINEARMAP: {
      const T v[6] = {p.x, p.px, p.y, p.py, p.zeta, p.ptau};
      T o[6];
      for (int i = 0; i < 6; i++) {
        T acc = mkv<T>(q.d[i]);
        for (int j = 0; j < 6; j++) acc = acc + q.M[6 * i + j] * v[j];
        o[i] = acc;
      }
      p.x = o[0]; p.px = o[1]; p.y = o[2]; p.py = o[3]; p.zeta = o[4]; p.ptau = o[5];
      energy_update(p, rc);
      break;
    }
    case T_APERTURE: {
      // Circular aperture: lost if x^2 + y^2 > r^2 (a point on the circle
      // survives) or if x or y is not finite.
      const double x = val(p.x), y = val(p.y);
      if (!(x * x + y * y <= q.r2)) {
        const bool fin = std::isfinite(x) && std::isfinite(y);
        mark_lost(p, fin ? 0 : -1, turn, elem);
      }
      break;
    }
    // Misalignments and tilts as changes of the reference system (section
    // "Lattice modelling and single particle tracking"): the new frame is
    // displaced by (dx, dy), or rotated by theta about the reference orbit,
    // x' = x cos + y sin, y' = -x sin + y cos, the same for (px, py).
    case T_XYSHIFT:
      p.x = p.x - q.dx;
      p.y = p.y - q.dy;
      break;
    case T_SROTATION: {
      const T x = p.x, y = p.y, px = p.px, py = p.py;
      p.x = q.cs * x + q.sn * y;
      p.y = q.cs * y - q.sn * x;
      p.px = q.cs * px + q.sn * py;
      p.py = q.cs * py - q.sn * px;
      break;
    }
    case T_QUAD: thick_quad(p, q.k1, q.Lq, rc); break;
    case T_BEND:
      if (q.bfull && q.bk1 != 0.0) bend_full_gradient(p, q.bk0, q.bh, q.bL, q.bk1, q.bn, rc, turn, elem);
      else if (q.bfull) bend_full(p, q.bk0, q.bh, q.bL, rc, turn, elem);
      else bend_expanded(p, q.bk0, q.bh, q.bL, q.bk1, rc);
      break;
    // 4D weak-strong beam-beam (section "Beam-beam interactions") and frozen
    // space charge (section "Space charge"): transverse kicks of a frozen
    // Gaussian charge.  Values only (the Jacobian entry points reject them).
    case T_BEAMBEAM4D:
    case T_SPACECHARGE: {
      double kx, ky;
      lens_kick(q, val(p.x), val(p.y), val(p.zeta), &kx, &ky);
      p.px = p.px + kx;
      p.py = p.py + ky;
      break;
    }
    // Rectangular aperture: lost unless xmin <= x <= xmax and ymin <= y <= ymax
    // (the boundary survives); a non-finite x or y is lost with state -1.
    case T_APERTURE_RECT: {
      const double x = val(p.x), y = val(p.y);
      if (!(x >= q.xmin && x <= q.xmax && y >= q.ymin && y <= q.ymax)) {
        const bool fin = std::isfinite(x) && std::isfinite(y);
        mark_lost(p, fin ? 0 : -1, turn, elem);
      }
      break;
    }
    // Elliptic aperture with semi-axes a, b: lost if (x/a)^2 + (y/b)^2 > 1.
    case T_APERTURE_ELLIPSE: {
      const double x = val(p.x), y = val(p.y);
      if (!(x * x * q.ia2 + y * y * q.ib2 <= 1.0)) {
        const bool fin = std::isfinite(x) && std::isfinite(y);
        mark_lost(p, fin ? 0 : -1, turn, elem);
      }
      break;
    }
    default: break;
  }
}

// End-of-turn guard: |x| or |y| above 1 m (or not finite) is lost (code -3)
// at the last element of the turn.
template <class T>
static inline void turn_guard(Part<T>& p, int turn, int n_el) {
  if (!(std::fabs(val(p.x)) <= 1.0 && std::fabs(val(p.y)) <= 1.0)) mark_lost(p, -3, turn, n_el - 1);
}

// ---------------------------------------------------------------------------
// Loss-location refinement (section "Particle-matter interaction and
// collimation studies": backtracking plus a polygonal interpolation of the
// aperture between two aperture elements).

// Reference frame at the entrance of a row: local = R(th) (lab - d), with
// R(th) (x, y) = (x cos + y sin, -x sin + y cos); built up from the shift and
// rotation rows before it.
struct Frame { double th, dx, dy; };

static bool is_aperture(int t) { return t == T_APERTURE || t == T_APERTURE_RECT || t == T_APERTURE_ELLIPSE; }

// Distance from the aperture's frame origin to its boundary along the ray at
// angle phi; negative if the origin is not strictly inside.
static double ray_to_boundary(const Element& e, double phi) {
  const double c = std::cos(phi), s = std::sin(phi);
  if (e.type == T_APERTURE) return e.p[0];
  if (e.type == T_APERTURE_ELLIPSE) {
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

// Crossing-number test of (x, y) against the polygon interpolated at weight
// w between polygons A and B (n vertices each, x then y per vertex).
static bool inside_polygon(double x, double y, const double* A, const double* B, double w, int n) {
  bool in = false;
  for (int k = 0; k < n; k++) {
    const int k2 = (k + 1 == n) ? 0 : k + 1;
    const double ax = A[2 * k] + w * (B[2 * k] - A[2 * k]);
    const double ay = A[2 * k + 1] + w * (B[2 * k + 1] - A[2 * k + 1]);
    const double bx = A[2 * k2] + w * (B[2 * k2] - A[2 * k2]);
    const double by = A[2 * k2 + 1] + w * (B[2 * k2 + 1] - A[2 * k2 + 1]);
    if ((ay > y) != (by > y)) {
      const double xi = ax + (y - ay) * (bx - ax) / (by - ay);
      if (x < xi) in = !in;
    }
  }
  return in;
}

// Inverse of one row's map (radiation off).  Returns false if the row has
// no inverse here (linear map, non-linear edge) or the backward drift is not
// defined.
static bool inverse_row(Part<double>& p, const Prep& q, const RefConst& rc) {
  switch (q.type) {
    case T_DRIFT:
      drift(p, -q.L, rc, 0, 0);
      return p.state == 1;
    case T_MULTIPOLE: {
      // the kick leaves x, y and delta unchanged: recompute it and take it back
      double fr, fi;
      multipole_field(p, q.m, &fr, &fi);
      if (q.m.hxl != 0.0) {
        p.zeta = p.zeta + q.m.hxl * p.x / p.rvv;
        p.px = p.px + q.m.k0h * p.x;
        p.px = p.px - ((q.m.hxl - q.m.c[0]) + q.m.hxl * p.delta);
      } else {
        p.px = p.px + q.m.c[0];
      }
      p.px = p.px + fr;
      p.py = p.py - (fi + q.m.s[0]);
      return true;
    }
    case T_CAVITY: {
      const double phi = q.lagr - q.krf * p.zeta;
      p.ptau = p.ptau - q.qv * std::sin(phi);
      energy_update(p, rc);
      return true;
    }
    case T_DIPEDGE:
      if (q.enl) return false;
      p.px = p.px - q.r21 * p.x;
      p.py = p.py - q.r43 * p.y;
      return true;
    case T_LINEARMAP: return false;
    case T_QUAD: thick_quad(p, q.k1, -q.Lq, rc); return true;
    case T_BEND:
      if (q.bfull && q.bk1 != 0.0) bend_full_gradient(p, q.bk0, q.bh, -q.bL, q.bk1, q.bn, rc, 0, 0);
      else if (q.bfull) bend_full(p, q.bk0, q.bh, -q.bL, rc, 0, 0);
      else bend_expanded(p, q.bk0, q.bh, -q.bL, q.bk1, rc);
      return p.state == 1;
    case T_BEAMBEAM4D:
    case T_SPACECHARGE: {  // x, y, zeta unchanged by the kick: take the same kick back
      double kx, ky;
      lens_kick(q, p.x, p.y, p.zeta, &kx, &ky);
      p.px = p.px - kx;
      p.py = p.py - ky;
      return true;
    }
    case T_XYSHIFT:
      p.x = p.x + q.dx;
      p.y = p.y + q.dy;
      return true;
    case T_SROTATION: {
      const double x = p.x, y = p.y, px = p.px, py = p.py;
      p.x = q.cs * x - q.sn * y;
      p.y = q.cs * y + q.sn * x;
      p.px = q.cs * px - q.sn * py;
      p.py = q.cs * py + q.sn * px;
      return true;
    }
    default: return true;  // markers, apertures
  }
}
}  // namespace xo

using namespace xo;

extern "C" {

// A table row the oracle accepts: a known type, a multipole order 0..10, a
// bend model 0 (expanded) or 1 (full) with 0..64 gradient kicks, an edge
// model 0 (linear), 1 (non-linear) or 2 (exact wedge) on face 0 or 1.
static bool row_ok(const Element& e) {
  if (e.type < 0 || e.type > T_SPACECHARGE) return false;
  if (e.type == T_MULTIPOLE && (e.order < 0 || e.order > 10)) return false;
  if (e.type == T_BEND && !(e.p[4] == 0.0 || e.p[4] == 1.0)) return false;
  if (e.type == T_DIPEDGE && !((e.p[4] == 0.0 || e.p[4] == 1.0 || e.p[4] == 2.0) && (e.p[5] == 0.0 || e.p[5] == 1.0)))
    return false;
  if (e.type == T_BEND && !(e.p[5] >= 0.0 && e.p[5] <= 64.0 && e.p[5] == std::floor(e.p[5]))) return false;
  return true;
}

// Reference length of a row (drift, thick quadrupole and thick bend).
static double row_length(const Element& e) {
  if (e.type == T_DRIFT) return e.p[0];
  if (e.type == T_QUAD) return e.p[1];
  if (e.type == T_BEND) return e.p[2];
  return 0.0;
}

// Tracks n particles (SoA arrays, updated in place) through n_turns turns of
// the lattice, starting at absolute turn start_turn.  rad_mode: 0 off, 1 mean,
// 2 quantum (Philox4x64-10 keyed by seed).  Particles with state != 1 on entry
// are left untouched.  Lost particles keep their coordinates at the loss point
// and record state, at_turn (absolute, 0-based) and at_element; survivors get
// at_turn = start_turn + n_turns, at_element = 0.  Returns 0, or -1 on an
// invalid argument.
int xo_track(const Element* el, int64_t n_el, const Reference* ref, int rad_mode, uint64_t seed,
             double* x, double* px, double* y, double* py, double* zeta, double* delta,
             double* ptau, double* rpp, double* rvv, int32_t* state, int32_t* at_turn,
             int32_t* at_element, const int64_t* pid, int64_t n, int64_t start_turn,
             int64_t n_turns) {
  if (!el || !ref || n_el <= 0 || n < 0 || n_turns < 0 || rad_mode < 0 || rad_mode > 2) return -1;
  const RefConst rc = ref_const(*ref);
  std::vector<Prep> prep(n_el);
  for (int64_t e = 0; e < n_el; e++) {
    if (!row_ok(el[e])) return -1;
    prep[e] = prepare(el[e], rc);
  }
  for (int64_t i = 0; i < n; i++) {
    Part<double> p;
    p.x = x[i]; p.px = px[i]; p.y = y[i]; p.py = py[i]; p.zeta = zeta[i];
    p.delta = delta[i]; p.ptau = ptau[i]; p.rpp = rpp[i]; p.rvv = rvv[i];
    p.state = state[i]; p.at_turn = at_turn[i]; p.at_element = at_element[i]; p.id = pid[i];
    if (p.state != 1) continue;
    for (int64_t t = start_turn; t < start_turn + n_turns && p.state == 1; t++) {
      for (int64_t e = 0; e < n_el; e++) {
        track_element(p, prep[e], rad_mode, rc, seed, (int)t, (int)e);
        if (p.state != 1) break;
      }
      if (p.state == 1) turn_guard(p, (int)t, (int)n_el);
    }
    if (p.state == 1) { p.at_turn = (int32_t)(start_turn + n_turns); p.at_element = 0; }
    x[i] = p.x; px[i] = p.px; y[i] = p.y; py[i] = p.py; zeta[i] = p.zeta;
    delta[i] = p.delta; ptau[i] = p.ptau; rpp[i] = p.rpp; rvv[i] = p.rvv;
    state[i] = p.state; at_turn[i] = p.at_turn; at_element[i] = p.at_element;
  }
  return 0;
}

// Loss-location refinement of the particles with state 0 lost at an aperture
// row (see the helpers above): s_loss[i] = position [m from the start of the
// table] where the trajectory first leaves the polygon interpolated between
// the previous aperture and the losing one, found by backtracking to the
// previous aperture and re-tracking with drifts cut into steps <= ds; the
// aperture's own position if no step is outside; NaN for other particles, a
// linear map in between, or an aperture whose frame origin is not inside it.
// Returns 0, or -1 on bad input.
int xo_refine_losses(const Element* el, int64_t n_el, const Reference* ref, const double* x, const double* px,
                     const double* y, const double* py, const double* zeta, const double* delta,
                     const double* ptau, const double* rpp, const double* rvv, const int32_t* state,
                     const int32_t* at_element, int64_t n, double ds, int n_angles, double* s_loss) {
  if (!el || !ref || n_el <= 0 || n < 0 || !(ds > 0.0) || n_angles < 8 || n_angles > 1024) return -1;
  const RefConst rc = ref_const(*ref);
  std::vector<Prep> prep(n_el);
  std::vector<double> spos(n_el + 1, 0.0);
  std::vector<Frame> fr(n_el);
  Frame f = {0.0, 0.0, 0.0};
  int64_t n_ap = 0;
  for (int64_t e = 0; e < n_el; e++) {
    if (!row_ok(el[e])) return -1;
    prep[e] = prepare(el[e], rc);
    fr[e] = f;
    spos[e + 1] = spos[e] + row_length(el[e]);
    if (el[e].type == T_XYSHIFT) {
      const double c = std::cos(f.th), sn = std::sin(f.th);
      f.dx = f.dx + (c * el[e].p[0] - sn * el[e].p[1]);
      f.dy = f.dy + (sn * el[e].p[0] + c * el[e].p[1]);
    } else if (el[e].type == T_SROTATION) {
      f.th = f.th + el[e].p[0];
    }
    if (is_aperture(el[e].type)) n_ap++;
  }
  if (n_ap == 0) return -1;
  const double C = spos[n_el];
  // laboratory-frame polygons of the apertures; previous aperture of each
  std::vector<std::vector<double>> poly(n_el);
  std::vector<int64_t> prev(n_el, -1);
  std::vector<char> ok(n_el, 0);
  const double two_pi = 6.283185307179586;
  int64_t last = -1;
  for (int64_t e = 0; e < n_el; e++)
    if (is_aperture(el[e].type)) last = e;
  for (int64_t e = 0; e < n_el; e++) {
    if (!is_aperture(el[e].type)) continue;
    prev[e] = last;
    last = e;
    poly[e].resize(2 * (size_t)n_angles);
    const double c = std::cos(fr[e].th), sn = std::sin(fr[e].th);
    ok[e] = 1;
    for (int k = 0; k < n_angles; k++) {
      const double phi = two_pi * (double)k / (double)n_angles;
      const double r = ray_to_boundary(el[e], phi);
      if (!(r > 0.0)) ok[e] = 0;
      const double lx = r * std::cos(phi), ly = r * std::sin(phi);
      poly[e][2 * k] = (c * lx - sn * ly) + fr[e].dx;
      poly[e][2 * k + 1] = (sn * lx + c * ly) + fr[e].dy;
    }
  }
  for (int64_t i = 0; i < n; i++) {
    s_loss[i] = NAN;
    const int64_t e = at_element[i];
    if (state[i] != 0 || e < 0 || e >= n_el || !is_aperture(el[e].type)) continue;
    const int64_t q = prev[e];
    if (!ok[e] || !ok[q]) continue;
    Part<double> p;
    p.x = x[i]; p.px = px[i]; p.y = y[i]; p.py = py[i]; p.zeta = zeta[i];
    p.delta = delta[i]; p.ptau = ptau[i]; p.rpp = rpp[i]; p.rvv = rvv[i];
    p.state = 1; p.at_turn = 0; p.at_element = 0; p.id = 0;
    // back to the exit of q
    bool good = true;
    for (int64_t j = e;;) {
      j = (j == 0) ? n_el - 1 : j - 1;
      if (j == q) break;
      if (!inverse_row(p, prep[j], rc)) { good = false; break; }
    }
    if (!good) continue;
    // forward again, drifts in steps, against the interpolated polygon
    const double s_q = spos[q];
    const double seg = (e > q) ? spos[e] - s_q : spos[e] + C - s_q;
    double pos = s_q;
    double found = NAN;
    for (int64_t j = q;;) {
      j = (j + 1 == n_el) ? 0 : j + 1;
      if (j == e) break;
      // drifts, thick quadrupoles and thick bends in steps of at most ds (the
      // thick maps are flows: their steps compose to the same map as one pass;
      // a full bend with a gradient is not, and is passed whole)
      const int ty = prep[j].type;
      const double L = row_length(el[j]);
      const bool kicked = ty == T_BEND && prep[j].bfull && prep[j].bk1 != 0.0;
      if ((ty == T_DRIFT || ty == T_QUAD || ty == T_BEND) && L > 0.0 && !kicked) {
        const int64_t ns = (int64_t)std::ceil(L / ds);
        const double h = L / (double)ns;
        const double c = std::cos(fr[j].th), sn = std::sin(fr[j].th);
        for (int64_t k = 1; k <= ns; k++) {
          if (ty == T_QUAD) thick_quad(p, prep[j].k1, h, rc);
          else if (ty == T_BEND && prep[j].bfull) bend_full(p, prep[j].bk0, prep[j].bh, h, rc, 0, 0);
          else if (ty == T_BEND) bend_expanded(p, prep[j].bk0, prep[j].bh, h, prep[j].bk1, rc);
          else drift(p, h, rc, 0, 0);
          const double at = pos + (double)k * h;
          if (p.state != 1) { found = at; break; }
          const double lx = (c * p.x - sn * p.y) + fr[j].dx;
          const double ly = (sn * p.x + c * p.y) + fr[j].dy;
          const double w = (at - s_q) / seg;
          if (!inside_polygon(lx, ly, poly[q].data(), poly[e].data(), w, n_angles)) { found = at; break; }
        }
        if (found == found) break;
        pos = pos + L;
      } else {
        track_element(p, prep[j], 0, rc, 0, 0, 0);
        if (p.state != 1) { found = pos; break; }
        if (kicked) pos = pos + L;
      }
    }
    if (!(found == found)) found = spos[e];
    s_loss[i] = (found >= C) ? found - C : found;
  }
  return 0;
}

// Differentiable tracking of one particle given in canonical coordinates
// z = (x, px, y, py, zeta, pzeta), pzeta = ptau/beta0, for n_turns turns
// (radiation 0 or 1).  Writes the final z and the Jacobian dz_out/dz_in
// (row-major 6x6).  If along != NULL it also receives, after every element of
// the first turn, 6 coordinates followed by the 36 Jacobian entries
// (n_el * 42 doubles).  Returns 0, 1 if the particle was lost, -1 on bad input.
int xo_track_jacobian(const Element* el, int64_t n_el, const Reference* ref, int rad_mode,
                      const double* z0, int64_t n_turns, double* z_out, double* M_out,
                      double* along) {
  if (!el || !ref || n_el <= 0 || rad_mode < 0 || rad_mode > 1) return -1;
  for (int64_t e = 0; e < n_el; e++)
    if (!row_ok(el[e]) || el[e].type == T_BEAMBEAM4D || el[e].type == T_SPACECHARGE) return -1;  // value-only
  const RefConst rc = ref_const(*ref);
  std::vector<Prep> prep(n_el);
  for (int64_t e = 0; e < n_el; e++) prep[e] = prepare(el[e], rc);
  Part<Dual> p;
  Dual* in[6] = {&p.x, &p.px, &p.y, &p.py, &p.zeta, &p.ptau};
  for (int k = 0; k < 6; k++) { *in[k] = mkd(z0[k]); in[k]->d[k] = 1.0; }
  p.ptau = p.ptau * rc.beta0;  // pzeta -> ptau
  p.state = 1; p.at_turn = 0; p.at_element = 0; p.id = 0;
  energy_update(p, rc);
  auto out6 = [&](double* zo, double* Mo) {
    Dual pz = p.ptau * rc.ib0;
    const Dual* o[6] = {&p.x, &p.px, &p.y, &p.py, &p.zeta, &pz};
    for (int i = 0; i < 6; i++) {
      zo[i] = o[i]->v;
      for (int j = 0; j < 6; j++) Mo[6 * i + j] = o[i]->d[j];
    }
  };
  for (int64_t t = 0; t < n_turns; t++) {
    for (int64_t e = 0; e < n_el; e++) {
      track_element(p, prep[e], rad_mode, rc, 0, (int)t, (int)e);
      if (p.state != 1) return 1;
      if (along && t == 0) out6(along + 42 * e, along + 42 * e + 6);
    }
  }
  out6(z_out, M_out);
  return 0;
}

// Closed orbit by Newton iteration on the one-turn map using the exact
// Jacobian.  dim = 6: fixed point of all six coordinates (needs RF);
// dim = 4: fixed point of (x,px,y,py) at the given pzeta (zeta is free).
// z is the initial guess and receives the orbit.  Returns the iteration count,
// or -1 on failure.
int xo_closed_orbit(const Element* el, int64_t n_el, const Reference* ref, int rad_mode, int dim,
                    double* z) {
  if (dim != 4 && dim != 6) return -1;
  for (int it = 0; it < 40; it++) {
    double zo[6], M[36];
    if (xo_track_jacobian(el, n_el, ref, rad_mode, z, 1, zo, M, nullptr) != 0) return -1;
    double A[6][7];
    double res = 0.0;
    for (int i = 0; i < dim; i++) {
      for (int j = 0; j < dim; j++) A[i][j] = M[6 * i + j] - (i == j ? 1.0 : 0.0);
      A[i][dim] = -(zo[i] - z[i]);
      res = std::max(res, std::fabs(zo[i] - z[i]));
    }
    if (res < 1e-15) return it;
    // Gaussian elimination with partial pivoting.
    for (int c = 0; c < dim; c++) {
      int piv = c;
      for (int r = c + 1; r < dim; r++) if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
      for (int k = 0; k <= dim; k++) std::swap(A[c][k], A[piv][k]);
      if (A[c][c] == 0.0) return -1;
      for (int r = c + 1; r < dim; r++) {
        double f = A[r][c] / A[c][c];
        for (int k = c; k <= dim; k++) A[r][k] -= f * A[c][k];
      }
    }
    double dz[6] = {0, 0, 0, 0, 0, 0};
    for (int r = dim - 1; r >= 0; r--) {
      double s = A[r][dim];
      for (int k = r + 1; k < dim; k++) s -= A[r][k] * dz[k];
      dz[r] = s / A[r][r];
    }
    for (int i = 0; i < dim; i++) z[i] += dz[i];
  }
  return -1;
}

// Chaos marker: finite-time Lyapunov estimate by the twin-particle method of
// Benettin, Galgani and Strelcyn (Phys. Rev. A 14, 2338 (1976)).  It tells
// regular orbits, whose neighbours separate at most linearly in the number of
// turns, from chaotic ones, where a separation grows exponentially and any
// rounding difference reaches the loss turn.
//
// Particle i starts at canonical z = (x, px, y, py, zeta, pzeta) (row i of
// z0, n x 6; pzeta = ptau/beta0), its twin at z + dz0.  Both are tracked turn
// by turn with the maps and loss checks of xo_track (radiation 0 or 1).
// After every `every` turns, and after the last one, the separation
// d = |A (z_twin - z)| is measured in the metric A (6 x 6 row-major, the
// identity if NULL); ln(d / d0), d0 = |A dz0|, is added to sum_log[i] and the
// twin is moved back to distance d0 along the current separation.
// turns[i] = turns completed by both; lost[i] = 0 if both survived, 2 if
// both were lost in the same turn, 1 if only one of them was lost (or the
// separation stopped being finite and positive).  The estimate is
// lambda = sum_log / turns per turn.  Returns 0, or -1 on bad input.
int xo_lyapunov(const Element* el, int64_t n_el, const Reference* ref, int rad_mode,
                const double* z0, const double* dz0, const double* metric, int64_t n,
                int64_t n_turns, int64_t every, double* sum_log, int32_t* turns, int32_t* lost) {
  if (!el || !ref || !z0 || !dz0 || n_el <= 0 || n < 0 || n_turns < 0 || every < 1 ||
      rad_mode < 0 || rad_mode > 1)
    return -1;
  const RefConst rc = ref_const(*ref);
  std::vector<Prep> prep(n_el);
  for (int64_t e = 0; e < n_el; e++) {
    if (!row_ok(el[e])) return -1;
    prep[e] = prepare(el[e], rc);
  }
  double A[36];
  for (int k = 0; k < 36; k++) A[k] = metric ? metric[k] : (k % 7 == 0 ? 1.0 : 0.0);
  auto norm = [&](const double* v) {
    double s = 0.0;
    for (int r = 0; r < 6; r++) {
      double w = 0.0;
      for (int c = 0; c < 6; c++) w += A[6 * r + c] * v[c];
      s += w * w;
    }
    return std::sqrt(s);
  };
  auto set = [&](Part<double>& p, const double* z, int64_t id) {
    p.x = z[0]; p.px = z[1]; p.y = z[2]; p.py = z[3]; p.zeta = z[4];
    p.ptau = z[5] * rc.beta0;
    p.state = 1; p.at_turn = 0; p.at_element = 0; p.id = id;
    energy_update(p, rc);
  };
  auto get = [&](const Part<double>& p, double* z) {
    z[0] = p.x; z[1] = p.px; z[2] = p.y; z[3] = p.py; z[4] = p.zeta; z[5] = p.ptau * rc.ib0;
  };
  auto one_turn = [&](Part<double>& p, int64_t t) {
    for (int64_t e = 0; e < n_el && p.state == 1; e++) track_element(p, prep[e], rad_mode, rc, 0, (int)t, (int)e);
    if (p.state == 1) turn_guard(p, (int)t, (int)n_el);
  };
  const double d0 = norm(dz0);
  if (!(d0 > 0.0) || !std::isfinite(d0)) return -1;
  for (int64_t i = 0; i < n; i++) {
    double zp[6], zq[6];
    for (int k = 0; k < 6; k++) { zp[k] = z0[6 * i + k]; zq[k] = zp[k] + dz0[k]; }
    Part<double> p, q;
    set(p, zp, i);
    set(q, zq, i);
    double S = 0.0;
    int64_t t = 0;
    int32_t code = 0;
    while (t < n_turns) {
      one_turn(p, t);
      one_turn(q, t);
      if (p.state != 1 || q.state != 1) {
        code = (p.state != 1 && q.state != 1) ? 2 : 1;
        break;
      }
      t++;
      if (t % every == 0 || t == n_turns) {
        get(p, zp);
        get(q, zq);
        double dv[6];
        for (int k = 0; k < 6; k++) dv[k] = zq[k] - zp[k];
        const double d = norm(dv);
        if (!(d > 0.0) || !std::isfinite(d)) { code = 1; break; }
        S += std::log(d / d0);
        for (int k = 0; k < 6; k++) zq[k] = zp[k] + dv[k] * (d0 / d);
        set(q, zq, i);
      }
    }
    sum_log[i] = S;
    turns[i] = (int32_t)t;
    lost[i] = code;
  }
  return 0;
}

// Test hooks for the building blocks.
void xo_philox4x64_10(const uint64_t* ctr, const uint64_t* key, uint64_t* out) { philox4x64_10(ctr, key, out); }
double xo_uniform(uint64_t seed, uint64_t pid, uint64_t turn, uint64_t elem, int64_t index) {
  Uniforms U(seed, pid, turn, elem);
  double u = 0.0;
  for (int64_t k = 0; k <= index; k++) u = U.next();
  return u;
}
int xo_spectrum_size(void) { return SPEC_K; }
void xo_spectrum_table(double* xi, double* F) {
  const Spectrum& S = spectrum();
  for (int i = 0; i < SPEC_K; i++) { xi[i] = S.xi[i]; F[i] = S.F[i]; }
}
double xo_spectrum_sample(double u) { return spectrum().sample(u); }
// Reference-derived constants, for tests: E0, beta0, gamma0, crad, kq, uc15.
void xo_ref_constants(const Reference* ref, double* out) {
  RefConst c = ref_const(*ref);
  out[0] = c.E0; out[1] = c.beta0; out[2] = c.gamma0; out[3] = c.crad; out[4] = c.kq; out[5] = c.uc15;
}
// Field shape of a unit bi-Gaussian line charge (sigma_x, sigma_y) at (x, y).
void xo_gauss_field(double sx, double sy, const double* x, const double* y, double* fx, double* fy, int64_t n) {
  for (int64_t i = 0; i < n; i++) gauss_field(x[i], y[i], sx, sy, &fx[i], &fy[i]);
}
// Nodes and weights of the quadrature rule on [-1, 1]; returns their number.
int xo_gauss_legendre(double* x, double* w) {
  const GaussLegendre& g = gauss_legendre();
  for (int i = 0; i < GaussLegendre::N; i++) { x[i] = g.x[i]; w[i] = g.w[i]; }
  return GaussLegendre::N;
}
// The entire functions of the thick maps at z: C, S, S2, S3 (for their pins).
void xo_osc_funcs(const double* z, double* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) osc_funcs(z[i], &out[4 * i], &out[4 * i + 1], &out[4 * i + 2], &out[4 * i + 3]);
}

}  // extern "C"
