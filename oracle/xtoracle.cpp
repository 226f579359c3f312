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
// and compensation").  The maps below are the textbook thin-lens Hamiltonian
// maps with MAD-X sign conventions; every operation order and every explicit
// fma is part of the map definition, so the CUDA path can reproduce the same
// bits.  Build with -O2 -ffp-contract=off (no implicit contraction).
//
// Coordinates: x, px=Px/P0, y, py, zeta=s-beta0*c*t, delta=(P-P0)/P0,
// ptau=(E-E0)/(P0 c), rpp=1/(1+delta), rvv=beta/beta0.
//
// The scalar type is a template parameter so the same map code yields values
// (double) and exact first derivatives (Dual, forward-mode differentiation)
// for the one-turn Jacobian, the closed orbit and the optics pins.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

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

// fma: one rounding for the value; exact derivative of a*b+c.
static inline double FMA(double a, double b, double c) { return std::fma(a, b, c); }
static inline Dual FMA(const Dual& a, const Dual& b, const Dual& c) {
  Dual r; r.v = std::fma(a.v, b.v, c.v);
  for (int i = 0; i < 6; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i] + c.d[i];
  return r;
}
static inline Dual FMA(double a, const Dual& b, const Dual& c) { return FMA(mkd(a), b, c); }
static inline Dual FMA(const Dual& a, double b, const Dual& c) { return FMA(a, mkd(b), c); }
static inline Dual FMA(const Dual& a, const Dual& b, double c) { return FMA(a, b, mkd(c)); }
static inline Dual FMA(double a, const Dual& b, double c) { return FMA(mkd(a), b, mkd(c)); }
static inline Dual FMA(const Dual& a, double b, double c) { return FMA(a, mkd(b), mkd(c)); }
// a b + c with a, b constants (used only by value-only elements)
static inline Dual FMA(double a, double b, const Dual& c) { Dual r = c; r.v = std::fma(a, b, c.v); return r; }
static inline double SQRT(double a) { return std::sqrt(a); }
static inline Dual SQRT(const Dual& a) { Dual r; r.v = std::sqrt(a.v); for (int i = 0; i < 6; i++) r.d[i] = a.d[i] / (2.0 * r.v); return r; }

// ---------------------------------------------------------------------------
// sin(x): Cody & Waite (1980) additive range reduction by pi/2 with a
// three-part constant, then the Taylor series of sin/cos on |r| <= pi/4
// evaluated by Horner's rule.  Written out so that both implementations of the
// tracker produce identical bits (library sin routines differ by an ulp).
// Valid for |x| < 2^40; accuracy about 1 ulp on |x| < 1e6.
static const double PIO2_1 = 1.5707963267948965579989817342720925807952880859375;
static const double PIO2_2 = 6.123233995736766035868820147291818682e-17;
static const double PIO2_3 = -1.4973849048591698329435081771059e-33;
static const double TWO_OVER_PI = 0.63661977236758134307553505349005744813783858296183;
static const double RND_MAGIC = 6755399441055744.0;  // 1.5 * 2^52

struct SinCoef {
  double s[10];  // (-1)^k / (2k+1)!, k = 0..9  (1, -1/3!, ..., -1/19!)
  double c[11];  // (-1)^k / (2k)!,  k = 0..10 (1, -1/2!, ..., 1/20!)
  SinCoef() {
    double f = 1.0;  // running factorial, exact up to 20! as a double
    for (int n = 1; n <= 21; n++) {
      f = f * (double)n;
      if (n % 2 == 1) { int k = (n - 1) / 2; if (k < 10) s[k] = ((k % 2) ? -1.0 : 1.0) / f; }
      else { int k = n / 2; if (k < 11) c[k] = ((k % 2) ? -1.0 : 1.0) / f; }
    }
    s[0] = 1.0; c[0] = 1.0;
  }
};
static const SinCoef SC;

double sin_cw(double x) {
  double k = (x * TWO_OVER_PI + RND_MAGIC) - RND_MAGIC;  // nearest integer
  double r = std::fma(-k, PIO2_1, x);
  r = std::fma(-k, PIO2_2, r);
  r = std::fma(-k, PIO2_3, r);
  long long q = (long long)k;
  int quad = (int)(q & 3);
  double z = r * r;
  double res;
  if (quad & 1) {  // cos r
    double p = SC.c[10];
    for (int i = 9; i >= 0; i--) p = std::fma(p, z, SC.c[i]);
    res = p;
  } else {  // sin r = r * (s0 + z*(s1 + ...))
    double p = SC.s[9];
    for (int i = 8; i >= 1; i--) p = std::fma(p, z, SC.s[i]);
    res = std::fma(r * z, p, r);
  }
  return (quad & 2) ? -res : res;
}
// cos x: the same reduction as sin_cw with the quadrant advanced by one.
double cos_cw(double x) {
  double k = (x * TWO_OVER_PI + RND_MAGIC) - RND_MAGIC;
  double r = std::fma(-k, PIO2_1, x);
  r = std::fma(-k, PIO2_2, r);
  r = std::fma(-k, PIO2_3, r);
  long long q = (long long)k;
  int quad = (int)((q + 1) & 3);
  double z = r * r;
  double res;
  if (quad & 1) {
    double p = SC.c[10];
    for (int i = 9; i >= 0; i--) p = std::fma(p, z, SC.c[i]);
    res = p;
  } else {
    double p = SC.s[9];
    for (int i = 8; i >= 1; i--) p = std::fma(p, z, SC.s[i]);
    res = std::fma(r * z, p, r);
  }
  return (quad & 2) ? -res : res;
}
static inline double SIN(double a) { return sin_cw(a); }
static inline double COS(double a) { return cos_cw(a); }
static inline Dual COS(const Dual& a) {
  Dual r; r.v = cos_cw(a.v); double sn = std::sin(a.v);
  for (int i = 0; i < 6; i++) r.d[i] = -sn * a.d[i];
  return r;
}
static inline Dual SIN(const Dual& a) {
  Dual r; r.v = sin_cw(a.v); double c = std::cos(a.v);
  for (int i = 0; i < 6; i++) r.d[i] = c * a.d[i];
  return r;
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based RNG.
// Counter = (particle id, turn, element index, call index); key = (seed, 0).
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
// 53-bit uniform in [0, 1) from a 64-bit word.
static inline double u01(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }

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
// the strip |Im t| < pi/2, so the rule converges geometrically).
static const int SPEC_K = 2048, SPEC_GUIDE = 4096;
static const double SPEC_XI_MIN = 1e-7, SPEC_XI_MAX = 40.0;
struct Spectrum {
  double xi[SPEC_K], F[SPEC_K];
  int guide[SPEC_GUIDE];  // guide[j] = max{i : F[i] <= j / SPEC_GUIDE} (Chen and Asau, 1974)
  double idF[SPEC_K];     // 1 / (F[i+1] - F[i]): the interpolation multiplies instead of dividing
  double iF0;             // 1 / F[0]
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
    int i = 0;
    for (int j = 0; j < SPEC_GUIDE; j++) {
      const double t = (double)j / (double)SPEC_GUIDE;
      while (i + 1 < SPEC_K && F[i + 1] <= t) i++;
      guide[j] = i;
    }
    for (int k = 0; k + 1 < SPEC_K; k++) idF[k] = 1.0 / (F[k + 1] - F[k]);
    idF[SPEC_K - 1] = 0.0;
    iF0 = 1.0 / F[0];
  }
  // Inverse CDF: power-law asymptote F ~ xi^(1/3) below the first knot,
  // linear interpolation between knots lo and lo + 1 with
  // lo = max{i : F[i] <= u} (walked up from the guide entry of u's cell),
  // clamp above the last knot.
  double sample(double u) const {
    if (u < F[0]) { double q = u * iF0; return xi[0] * q * q * q; }
    if (u >= F[SPEC_K - 1]) return xi[SPEC_K - 1];
    int lo = guide[(int)(u * (double)SPEC_GUIDE)];
    while (F[lo + 1] <= u) lo++;
    const int hi = lo + 1;
    double w = (u - F[lo]) * idF[lo];
    return xi[lo] + w * (xi[hi] - xi[lo]);
  }
};
static const Spectrum& spectrum() { static Spectrum s; return s; }

// ---------------------------------------------------------------------------
// Reference-derived constants (computed once per call on the host).
struct RefConst {
  double m0, q0, p0c, E0, beta0, gamma0, bg0, ib0, twoib0;
  // radiation
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
  const double rc = r.q0 * r.q0 * R_ELECTRON * M_ELECTRON / r.mass0;
  c.crad = 2.0 * rc * r.mass0 / (3.0 * r.p0c);
  c.kq = 5.0 * ALPHA_FS * r.q0 * r.q0 / (2.0 * std::sqrt(3.0));
  c.uc15 = 1.5 * HBAR_C;
  return c;
}

// ---------------------------------------------------------------------------
// Special functions of the beam-beam kick (section "Beam-beam interactions").

// 1/n! for n = 0..21 (n! is exact in double up to 18!; beyond, the running
// product rounds, far below what the series that use these terms resolve).
static const std::vector<double>& inv_fact() {
  static std::vector<double> c = [] {
    std::vector<double> v(22);
    double f = 1.0;
    for (int n = 0; n <= 21; n++) {
      if (n > 0) f = f * (double)n;
      v[n] = 1.0 / f;
    }
    return v;
  }();
  return c;
}

// e^x: Cody-Waite reduction x = k ln2 + r with ln 2 split into a head with
// 20 significant bits (k * head exact) and a tail, e^r by its Taylor series
// to r^13 on |r| <= ln2/2 (truncation below 1e-17 relative), times 2^k from
// the exponent bits (in two steps below the normal range).
static double exp_cw(double x) {
  if (x != x) return x;
  if (!(x > -745.2)) return 0.0;
  if (x > 709.7) return INFINITY;
  const double sh = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer
  const double t = std::fma(x, 1.4426950408889634, sh) - sh;
  const int k = (int)t;
  double r = std::fma(-t, 0x1.62e42p-1, x);
  r = std::fma(-t, 0x1.fdf473de6af28p-22, r);
  const std::vector<double>& c = inv_fact();
  double p = c[13];
  for (int n = 12; n >= 0; n--) p = std::fma(p, r, c[n]);
  auto pow2 = [](int e) {
    const uint64_t b = (uint64_t)(e + 1023) << 52;
    double v;
    std::memcpy(&v, &b, 8);
    return v;
  };
  if (k >= -1022) return p * pow2(k);
  return (p * pow2(k + 64)) * pow2(-64);
}

// 1 - e^(-u) for u >= 0 without cancellation: for u < 1/2 the series
// u sum_n (-u)^n / (n+1)!, n = 0..17 (truncation below 1e-22), else 1 - e^(-u).
static double one_minus_exp(double u) {
  const std::vector<double>& c = inv_fact();
  if (u < 0.5) {
    double s = c[18];
    for (int n = 16; n >= 0; n--) s = std::fma(s, -u, c[n + 1]);
    return u * s;
  }
  return 1.0 - exp_cw(-u);
}

// e^a for scalars and dual numbers (the hyperbolic branch of the oscillator
// functions of the thick elements).
static inline double EXPC(double a) { return exp_cw(a); }
static inline Dual EXPC(const Dual& a) {
  Dual r; r.v = exp_cw(a.v);
  for (int i = 0; i < 6; i++) r.d[i] = r.v * a.d[i];
  return r;
}

// Faddeeva function w(z) = e^(-z^2) erfc(-i z) for Im z >= 0 by Weideman's
// rational expansion (J. A. C. Weideman, SIAM J. Numer. Anal. 31 (1994)
// 1497): w = 2 p(Z) / (L - i z)^2 + (1/sqrt(pi)) / (L - i z), Z = (L + i z) /
// (L - i z), p a polynomial of degree N - 1 = 39, L = (N / sqrt 2)^(1/2);
// p's coefficients are the cosine transform of e^(-t^2)(L^2 + t^2) sampled at
// t = L tan(theta/2), here by a plain DFT.
struct Faddeeva {
  double L;
  double a[40];  // p(Z) = sum_n a[n] Z^n
};
static const Faddeeva& faddeeva_coefficients() {
  static Faddeeva c = [] {
    Faddeeva q;
    const int N = 40, M = 2 * N, M2 = 2 * M;
    const double L = std::sqrt((double)N / std::sqrt(2.0));
    std::vector<double> f(M2), fs(M2);
    f[0] = 0.0;
    for (int j = 1; j < M2; j++) {
      const int k = j - M;  // -M+1 .. M-1
      const double theta = (double)k * PI / (double)M;
      const double t = L * std::tan(theta / 2.0);
      f[j] = std::exp(-t * t) * (L * L + t * t);
    }
    for (int j = 0; j < M2; j++) fs[j] = f[(j + M) % M2];
    q.L = L;
    for (int n = 0; n < N; n++) {
      const int m = n + 1;
      double acc = 0.0;
      for (int j = 0; j < M2; j++) acc = acc + fs[j] * std::cos(2.0 * PI * (double)((j * m) % M2) / (double)M2);
      q.a[n] = acc / (double)M2;
    }
    return q;
  }();
  return c;
}

static void faddeeva(double x, double y, double* wr, double* wi) {
  const Faddeeva& c = faddeeva_coefficients();
  const double L = c.L;
  const double cr = L + y;                      // L - i z = (L + y) - i x
  const double D = std::fma(cr, cr, x * x);
  const double qr = cr / D, qi = x / D;         // q = 1 / (L - i z)
  const double ar = L - y;                      // L + i z = (L - y) + i x
  const double Zr = std::fma(ar, qr, -(x * qi));
  const double Zi = std::fma(ar, qi, x * qr);
  double pr = c.a[39], pi = 0.0;
  for (int n = 38; n >= 0; n--) {
    const double nr = std::fma(pr, Zr, std::fma(-pi, Zi, c.a[n]));
    const double ni = std::fma(pr, Zi, pi * Zr);
    pr = nr;
    pi = ni;
  }
  const double tr = std::fma(pr, qr, -(pi * qi));  // t = p q
  const double ti = std::fma(pr, qi, pi * qr);
  const double ur = std::fma(2.0, tr, 0.5641895835477563);  // u = 2 p q + 1/sqrt(pi)
  const double ui = 2.0 * ti;
  *wr = std::fma(qr, ur, -(qi * ui));  // w = q u
  *wi = std::fma(qr, ui, qi * ur);
}

// Constants of a 4D beam-beam lens (table: p[0] = charge times number of
// particles of the strong bunch [e], p[1] = its speed beta_s (moving against
// the tracked beam), p[2], p[3] = sigma_x, sigma_y [m], p[4], p[5] = its
// centre [m]).
struct BBConst {
  double K, xc, yc;
  int mode;        // 0 round, 1 sigma_x > sigma_y, 2 sigma_y > sigma_x
  double h1, h2;   // 1/(2 sigma_1^2), 1/(2 sigma_2^2) (round: h1 = 1/(2 sigma^2))
  double rs, rsi;  // sigma_2/sigma_1, sigma_1/sigma_2
  double invS, cpre;  // 1/S, sqrt(pi)/S, S = sqrt(2 (sigma_1^2 - sigma_2^2))
  double lin1, lin2;  // 1/(sigma_1 (sigma_1 + sigma_2)), 1/(sigma_2 (sigma_1 + sigma_2))
};

// Field of a unit bi-Gaussian line charge, f = E 2 pi eps0 / lambda, at (x, y)
// about its centre: Bassetti-Erskine with w(z) in the first quadrant and the
// signs restored from symmetry; round beam: (x, y)(1 - e^(-r^2/2 sigma^2))/r^2.
// Within rho^2 = (x/sigma_x)^2 + (y/sigma_y)^2 < 1e-10 of the centre the
// difference of the two w values cancels, and the linear field
// (x / (sigma_x (sigma_x + sigma_y)), y / (sigma_y (sigma_x + sigma_y))),
// whose relative error there is of order rho^2, is used instead.
static void gauss_field(double x, double y, const BBConst& b, double* fx, double* fy) {
  const double ax = std::fabs(x), ay = std::fabs(y);
  double gx, gy;
  if (b.mode == 0) {
    const double r2 = std::fma(ax, ax, ay * ay);
    const double g = (r2 == 0.0) ? b.h1 : one_minus_exp(r2 * b.h1) / r2;
    gx = ax * g;
    gy = ay * g;
  } else {
    const double u = (b.mode == 1) ? ax : ay, v = (b.mode == 1) ? ay : ax;  // u along the larger sigma
    const double h = std::fma(u, u * b.h1, v * (v * b.h2));                // rho^2 / 2
    double fu, fv;
    if (h < 5e-11) {
      fu = u * b.lin1;
      fv = v * b.lin2;
    } else {
      double w1r, w1i, w2r, w2i;
      faddeeva(u * b.invS, v * b.invS, &w1r, &w1i);
      faddeeva((u * b.rs) * b.invS, (v * b.rsi) * b.invS, &w2r, &w2i);
      const double e = exp_cw(-h);
      fu = b.cpre * std::fma(-e, w2i, w1i);  // Im of (sqrt(pi)/S)(w1 - e w2)
      fv = b.cpre * std::fma(-e, w2r, w1r);  // Re
    }
    gx = (b.mode == 1) ? fu : fv;
    gy = (b.mode == 1) ? fv : fu;
  }
  *fx = std::copysign(gx, x);
  *fy = std::copysign(gy, y);
}

template <class T> static inline T mkv(double v);
template <> inline double mkv<double>(double v) { return v; }
template <> inline Dual mkv<Dual>(double v) { return mkd(v); }

// ---------------------------------------------------------------------------
// Particle state; opd = 1+delta, dm1 = (1+delta)^2 - 1 = delta (delta + 2),
// ep = 1 + beta0 ptau (= opd / rvv), rv0v = 1/rvv = ep rpp and
// epm1 = beta0 ptau are derived from delta, rpp and ptau and recomputed
// whenever those change (pure functions of the stored state, so
// recomputation never changes a result).
template <class T>
struct Part {
  T x, px, y, py, zeta, delta, ptau, rpp, rvv;
  T opd, dm1, rv0v, ep, epm1;
  int32_t state, at_turn, at_element;
  int64_t id;
};
template <class T>
static inline void derive(Part<T>& p, const RefConst& rc) {
  p.opd = 1.0 + p.delta;
  p.dm1 = p.delta * (p.delta + 2.0);
  p.ep = FMA(rc.beta0, p.ptau, 1.0);
  p.rv0v = p.ep * p.rpp;
  p.epm1 = rc.beta0 * p.ptau;
}

// Energy update from a new ptau, using (1+delta)^2 = 1 + 2 ptau/beta0 + ptau^2
// written in the cancellation-free form delta = u / (sqrt(1+u) + 1),
// u = ptau (ptau + 2/beta0); then rpp = 1/(1+delta),
// rvv = (1+delta)/(1 + beta0 ptau) and 1/rvv = (1 + beta0 ptau) rpp.
template <class T>
static inline void energy_update(Part<T>& p, const RefConst& rc) {
  T u = p.ptau * (p.ptau + rc.twoib0);
  T s = SQRT(1.0 + u);
  p.delta = u / (s + 1.0);
  p.opd = 1.0 + p.delta;
  p.dm1 = p.delta * (p.delta + 2.0);
  p.rpp = 1.0 / p.opd;
  p.ep = FMA(rc.beta0, p.ptau, 1.0);
  p.rvv = p.opd / p.ep;
  p.rv0v = p.ep * p.rpp;
  p.epm1 = rc.beta0 * p.ptau;
}

template <class T>
static inline void mark_lost(Part<T>& p, int code, int turn, int elem) {
  p.state = code; p.at_turn = turn; p.at_element = elem;
}

// Exact drift of length L (thin-lens integration: drifts between kicks).
//   pz = sqrt((1+delta)^2 - px^2 - py^2),  x += px L/pz,  y += py L/pz,
//   zeta += L - (1+delta)/rvv * L/pz  (path length L(1+delta)/pz at speed beta).
// With u = (1+delta)^2 - 1 - px^2 - py^2 (two fused multiply-adds from
// dm1 = delta (delta + 2)) and yh = 1/pz - 1 = (1+u)^(-1/2) - 1:
//   L/pz = L + L yh,   zeta += -L (beta0 ptau + ep yh)   (ep - 1 = beta0 ptau),
// so the zeta increment is formed from small quantities without cancellation.
// yh is the Taylor series of (1+u)^(-1/2) - 1 to order 8 (coefficients
// binomial(-1/2, n), exact dyadic numbers) for |u| <= 2^-7, where the
// truncation error is below 2e-17 of yh; otherwise 1/sqrt(1+u) - 1.
// A particle with u outside (-1, inf) is lost (code -2), coordinates unchanged.
// Taylor coefficients of (1+u)^(-1/2) - 1: binomial(-1/2, n), exact dyadics.
static const double RS_C[9] = {0.0, -0.5, 0.375, -0.3125, 0.2734375, -0.24609375, 0.2255859375,
                               -0.20947265625, 0.196380615234375};

// yh = (1+u)^(-1/2) - 1 for u in (-1, inf).  The Taylor series truncated at
// order n leaves c_{n+1} u^{n+1}, i.e. about 2 |c_{n+1}| |u|^n relative to
// yh ~ -u/2; the order is the lowest that keeps this below 2^-54 (half an
// ulp) on its interval: order 3 for |u| <= 2^-18, 6 for |u| <= 2^-9, 8 for
// |u| <= 2^-7 (Horner from the highest order, then times u); beyond that
// 1/sqrt(1+u) - 1.
template <class T>
static inline T inv_pz_m1(T u) {
  const double a = std::fabs(val(u));
  int order = 0;
  if (a <= 0x1p-18) order = 3;
  else if (a <= 0x1p-9) order = 6;
  else if (a <= 0x1p-7) order = 8;
  if (order == 0) return 1.0 / SQRT(1.0 + u) - 1.0;
  T h = mkv<T>(RS_C[order]);
  for (int n = order - 1; n >= 1; n--) h = FMA(h, u, mkv<T>(RS_C[n]));
  return h * u;
}

template <class T>
static inline void drift(Part<T>& p, double L, int turn, int elem) {
  T u = FMA(-p.px, p.px, FMA(-p.py, p.py, p.dm1));
  double uv = val(u);
  if (!(uv > -1.0 && uv < INFINITY)) { mark_lost(p, -2, turn, elem); return; }
  T yh = inv_pz_m1(u);
  T lpz = FMA(L, yh, mkv<T>(L));
  p.x = FMA(p.px, lpz, p.x);
  p.y = FMA(p.py, lpz, p.y);
  p.zeta = FMA(-L, FMA(p.ep, yh, p.epm1), p.zeta);
}

// Energy change by radiation: ptau += dpt, then the energy update; the
// transverse momenta are scaled by (1+delta_new)/(1+delta_old) so that the
// angles px/(1+delta), py/(1+delta) are unchanged (emission along the motion).
template <class T>
static inline void apply_energy_loss(Part<T>& p, T dpt, const RefConst& rc) {
  T rpp_old = p.rpp;
  p.ptau = p.ptau + dpt;
  energy_update(p, rc);
  T f = p.opd * rpp_old;
  p.px = p.px * f;
  p.py = p.py * f;
}

// Per-element host constants of a thin multipole: cn = knl_n/n!, sn = ksl_n/n!,
// k0h = knl0*hxl/L_rad (0 when L_rad == 0), ilr2 = 1/L_rad^2,
// crl = crad*L_rad, kql = kq*L_rad.
struct MultConst {
  int N;
  double c[11], s[11];
  double hxl, k0h, lrad, ilr2, crl, kql;
  bool pure;    // knl0 == ksl0 == 0 and hxl == 0: no constant term
  bool bend;    // hxl != 0, hxl == knl0, ksl0 == 0: field and frame curvature cancel on momentum
};

// Quantum model: Poisson number of photons with mean
// nbar = (5/(2 sqrt 3)) alpha q0^2 gamma h L, energies u = u_c xi with
// u_c = (3/2) hbar c gamma^3 h and xi drawn from the synchrotron spectrum.
static const int KMAX_PHOTONS = 200;
// 1/k for k = 0..KMAX_PHOTONS (entry 0 unused): the Poisson recurrence
// pk = pk nbar / k multiplies by it.
static const std::vector<double>& recip_k() {
  static std::vector<double> r = [] {
    std::vector<double> v(KMAX_PHOTONS + 1, 0.0);
    for (int k = 1; k <= KMAX_PHOTONS; k++) v[k] = 1.0 / (double)k;
    return v;
  }();
  return r;
}
static inline void quantum_kick(Part<double>& p, double br, double bi, const MultConst& m,
                                const RefConst& rc, uint64_t seed, int turn, int elem) {
  double kk = std::fma(br, br, bi * bi);
  double h = std::sqrt(kk * m.ilr2) * p.rpp;
  double gam = std::fma(rc.bg0, p.ptau, rc.gamma0);
  double nbar = (m.kql * gam) * h;
  Uniforms U(seed, (uint64_t)p.id, (uint64_t)turn, (uint64_t)elem);
  double u0 = U.next();
  int k = 0;
  double pk = exp_cw(-nbar), F = pk;
  const std::vector<double>& rk = recip_k();
  while (u0 > F && k < KMAX_PHOTONS) { k++; pk = (pk * nbar) * rk[k]; F = F + pk; }
  if (k == 0) return;
  const Spectrum& S = spectrum();
  double sxi = 0.0;
  for (int j = 0; j < k; j++) sxi = sxi + S.sample(U.next());
  double uc = (rc.uc15 * (gam * gam * gam)) * h;
  double dpt = -(uc * sxi) / rc.p0c;
  apply_energy_loss(p, dpt, rc);
}
static inline void quantum_kick(Part<Dual>&, const Dual&, const Dual&, const MultConst&,
                                const RefConst&, uint64_t, int, int) {}

// Thin multipole: b = sum_n (knl_n + i ksl_n) z^n / n!, z = x + i y, by
// Horner's rule from the highest order; px -= Re b, py += Im b.  With a
// curvature hxl: px += hxl (1+delta) - knl0 hxl x / L_rad and
// zeta -= hxl x / rvv (the thin dipole of the curved reference frame).
// Radiation (mode 1 mean, 2 quantum) is applied once, after the kick, for
// elements with L_rad > 0, using the field kick (Re b, Im b) only.  Without
// radiation, elements with no constant term, and bends whose curvature equals
// their dipole field, add the last Horner step straight into px, py.
template <class T>
static inline void multipole(Part<T>& p, const MultConst& m, int rad_mode, const RefConst& rc,
                             uint64_t seed, int turn, int elem) {
  const bool radiates = rad_mode != 0 && m.lrad > 0.0;
  if (!radiates && (m.pure || m.bend)) {
    // Folded form: with (ar, ai) the Horner value after the linear-term step,
    // Re b = ar x - ai y + knl0, Im b = ar y + ai x + ksl0; the constant terms
    // vanish (pure) or combine with the curvature term as
    // -knl0 + hxl (1+delta) = hxl delta (bend, hxl == knl0).
    T pxv = m.bend ? FMA(m.hxl, p.delta, p.px) : p.px;
    if (m.N >= 1) {
      T ar = mkv<T>(m.c[m.N]);
      T ai = mkv<T>(m.s[m.N]);
      for (int n = m.N - 1; n >= 1; n--) {
        T nr = FMA(ar, p.x, FMA(-ai, p.y, mkv<T>(m.c[n])));
        T ni = FMA(ar, p.y, FMA(ai, p.x, mkv<T>(m.s[n])));
        ar = nr; ai = ni;
      }
      pxv = FMA(-ar, p.x, FMA(ai, p.y, pxv));
      p.py = FMA(ar, p.y, FMA(ai, p.x, p.py));
    }
    p.px = pxv;
    if (m.bend) {
      p.px = FMA(-m.k0h, p.x, p.px);
      p.zeta = FMA(-(m.hxl * p.rv0v), p.x, p.zeta);
    }
    return;
  }
  T br = mkv<T>(m.c[m.N]);
  T bi = mkv<T>(m.s[m.N]);
  for (int n = m.N - 1; n >= 0; n--) {
    T nr = FMA(br, p.x, FMA(-bi, p.y, mkv<T>(m.c[n])));
    T ni = FMA(br, p.y, FMA(bi, p.x, mkv<T>(m.s[n])));
    br = nr; bi = ni;
  }
  p.px = p.px - br;
  p.py = p.py + bi;
  if (m.hxl != 0.0) {
    p.px = FMA(m.hxl, p.opd, p.px);
    p.px = FMA(-m.k0h, p.x, p.px);
    p.zeta = FMA(-(m.hxl * p.rv0v), p.x, p.zeta);
  }
  if (rad_mode == 1 && m.lrad > 0.0) {
    // Mean model: dE = -(2/3) r_c m0 c^2 beta^3 gamma^4 h^2 L_rad with the local
    // curvature h = |field kick| / ((1+delta) L_rad).
    T kk = FMA(br, br, bi * bi);
    T h2 = (kk * m.ilr2) * (p.rpp * p.rpp);
    T gam = FMA(rc.bg0, p.ptau, mkv<T>(rc.gamma0));
    T bet = rc.beta0 * p.rvv;
    T b3 = bet * bet * bet;
    T g2 = gam * gam;
    T g4 = g2 * g2;
    T dpt = (-m.crl) * b3 * g4 * h2;
    apply_energy_loss(p, dpt, rc);
  } else if (rad_mode == 2 && m.lrad > 0.0) {
    quantum_kick(p, br, bi, m, rc, seed, turn, elem);
  }
}

// Prepared element: host constants of each type.
struct Prep {
  int type;
  double L;                              // drift
  MultConst m;                           // multipole
  double krf, lagr, qv;                  // cavity
  double r21, r43;                       // dipole edge (linear model)
  int enl;                               // dipole edge: 1 = non-linear model
  double ek0, et, esg, ecorr;            // non-linear edge: field, tan(e1), +1 entrance / -1 exit,
                                         // finite-extent vertical correction
  double M[36], d[6];                    // linear map in (x,px,y,py,zeta,ptau)
  double r2;                             // aperture
  double dx, dy;                         // reference-frame shift
  double cs, sn;                         // reference-frame rotation about s
  double xmin, xmax, ymin, ymax;         // rectangular aperture
  double ia2, ib2;                       // elliptic aperture: 1/a^2, 1/b^2
  BBConst bb;                            // 4D beam-beam lens; frozen space charge (shape and K)
  double sc_i2sz2;                       // frozen space charge: 1/(2 sigma_z^2), 0 for a coasting beam
  double k1, Lq;                         // thick quadrupole
  double bk0, bh, bL, bk1;               // thick bend: field, curvature, length, gradient
  int bfull;                             // thick bend: 1 = full model, 0 = expanded
};

// Field-shape constants of a bi-Gaussian line charge with sigma_x, sigma_y
// (gauss_field): round when the two squares agree to 1e-10, else the
// Bassetti-Erskine constants with sigma_1 the larger.
static void gauss_shape(BBConst& b, double sx, double sy) {
  const double sx2 = sx * sx, sy2 = sy * sy;
  if (std::fabs(sx2 - sy2) <= 1e-10 * (sx2 + sy2)) {
    b.mode = 0;
    b.h1 = 1.0 / (sx2 + sy2);
  } else {
    const bool flat = sx2 > sy2;
    const double s1 = flat ? sx : sy, s2 = flat ? sy : sx;
    b.mode = flat ? 1 : 2;
    const double S = std::sqrt(2.0 * (s1 * s1 - s2 * s2));
    b.h1 = 1.0 / (2.0 * (s1 * s1));
    b.h2 = 1.0 / (2.0 * (s2 * s2));
    b.rs = s2 / s1;
    b.rsi = s1 / s2;
    b.invS = 1.0 / S;
    b.cpre = 1.772453850905516 / S;
    b.lin1 = 1.0 / (s1 * (s1 + s2));
    b.lin2 = 1.0 / (s2 * (s1 + s2));
  }
}

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
      q.m.ilr2 = (q.m.lrad > 0.0) ? 1.0 / (q.m.lrad * q.m.lrad) : 0.0;
      q.m.crl = rc.crad * q.m.lrad;
      q.m.kql = rc.kq * q.m.lrad;
      q.m.pure = (e.p[0] == 0.0 && e.p[11] == 0.0 && q.m.hxl == 0.0);
      q.m.bend = (q.m.hxl != 0.0 && q.m.hxl == e.p[0] && e.p[11] == 0.0);
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
      q.enl = (e.p[4] != 0.0);
      q.ek0 = h;
      q.et = std::tan(e1);
      q.esg = (e.p[5] != 0.0) ? -1.0 : 1.0;
      q.ecorr = q.r21 + q.r43;  // h tan(e1) - h tan(e1 - psi)
      break;
    }
    case T_LINEARMAP: {
      // The table gives M, d on (x,px,y,py,zeta,pzeta), pzeta = ptau/beta0;
      // convert to (..., ptau): row 5 times beta0, column 5 divided by beta0.
      for (int i = 0; i < 6; i++) {
        for (int j = 0; j < 6; j++) {
          double v = e.p[6 * i + j];
          if (i == 5 && j != 5) v = v * rc.beta0;
          else if (j == 5 && i != 5) v = v * rc.ib0;
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
    case T_BEND: q.bk0 = e.p[0]; q.bh = e.p[1]; q.bL = e.p[2]; q.bk1 = e.p[3]; q.bfull = (e.p[4] != 0.0); break;
    case T_BEAMBEAM4D: {
      // kick of a counter-moving Gaussian bunch integrated over the crossing:
      // Delta p_perp / P0 = 2 q0 q_s N_s (r_e m_e c^2 / p0 c) (1 + beta0 beta_s) /
      // (beta0 + beta_s) f(x - x_c, y - y_c)
      const double qN = e.p[0], bs = e.p[1];
      BBConst& b = q.bb;
      b.K = 2.0 * rc.q0 * qN * (R_ELECTRON * M_ELECTRON) / rc.p0c * ((1.0 + rc.beta0 * bs) / (rc.beta0 + bs));
      b.xc = e.p[4];
      b.yc = e.p[5];
      gauss_shape(b, e.p[2], e.p[3]);
      break;
    }
    case T_SPACECHARGE: {
      // frozen space charge (section "Space charge", frozen model): the beam's
      // own Gaussian line charge of peak density lambda0 [1/m], electric and
      // magnetic forces cancelling to 1/gamma^2, integrated over the length L
      // the lumped element stands for:
      // Delta p_perp / P0 = 2 r_c lambda0 L / (beta0^2 gamma0^3) g(zeta) f(x - x_c, y - y_c),
      // r_c = q0^2 r_e m_e / m0, g = exp(-zeta^2 / (2 sigma_z^2)) (1 when sigma_z = 0)
      const double lam0 = e.p[0], sz = e.p[1], L = e.p[4];
      const double rcl = rc.q0 * rc.q0 * R_ELECTRON * M_ELECTRON / rc.m0;
      BBConst& b = q.bb;
      b.K = 2.0 * rcl * lam0 * L / (rc.beta0 * rc.beta0 * rc.gamma0 * rc.gamma0 * rc.gamma0);
      b.xc = e.p[5];
      b.yc = e.p[6];
      gauss_shape(b, e.p[2], e.p[3]);
      q.sc_i2sz2 = (sz > 0.0) ? 1.0 / (2.0 * (sz * sz)) : 0.0;
      break;
    }
    default: break;
  }
  return q;
}

// One element.  Returns with p.state != 1 if the particle was lost here.
template <class T>
static inline void track_element(Part<T>& p, const Prep& q, int rad_mode, const RefConst& rc,
                                 uint64_t seed, int turn, int elem) {
  switch (q.type) {
    case T_DRIFT: drift(p, q.L, turn, elem); break;
    case T_MULTIPOLE: multipole(p, q.m, rad_mode, rc, seed, turn, elem); break;
    case T_CAVITY: {
      // Thin RF: phase lag - k zeta, k = 2 pi f/(beta0 c); energy gain q0 V sin(phase).
      T phi = FMA(-q.krf, p.zeta, mkv<T>(q.lagr));
      p.ptau = FMA(q.qv, SIN(phi), p.ptau);
      energy_update(p, rc);
      break;
    }
    case T_DIPEDGE:
      if (q.enl) {
        edge_nonlinear(p, q.ek0, q.et, q.esg, q.r21, q.ecorr, turn, elem);
      } else {
        p.px = FMA(q.r21, p.x, p.px);
        p.py = FMA(q.r43, p.y, p.py);
      }
      break;
    case T_LINEARMAP: {
      T v[6] = {p.x, p.px, p.y, p.py, p.zeta, p.ptau};
      T o[6];
      for (int i = 0; i < 6; i++) {
        T acc = mkv<T>(q.d[i]);
        for (int j = 0; j < 6; j++) acc = FMA(q.M[6 * i + j], v[j], acc);
        o[i] = acc;
      }
      p.x = o[0]; p.px = o[1]; p.y = o[2]; p.py = o[3]; p.zeta = o[4]; p.ptau = o[5];
      energy_update(p, rc);
      break;
    }
    case T_APERTURE: {
      // Circular aperture: lost if x^2 + y^2 > r^2 (a point on the circle
      // survives) or if x or y is not finite.
      T rr = FMA(p.x, p.x, p.y * p.y);
      if (!(val(rr) <= q.r2)) {
        bool fin = std::isfinite(val(p.x)) && std::isfinite(val(p.y));
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
      p.x = FMA(q.cs, x, q.sn * y);
      p.y = FMA(q.cs, y, -(q.sn * x));
      p.px = FMA(q.cs, px, q.sn * py);
      p.py = FMA(q.cs, py, -(q.sn * px));
      break;
    }
    case T_QUAD: thick_quad(p, q.k1, q.Lq); break;
    case T_BEND:
      if (q.bfull) bend_full(p, q.bk0, q.bh, q.bL, turn, elem);
      else bend_expanded(p, q.bk0, q.bh, q.bL, q.bk1);
      break;
    // 4D weak-strong beam-beam (section "Beam-beam interactions"): transverse
    // kick of a frozen Gaussian bunch, independent of the longitudinal
    // coordinates.  Values only (the Jacobian entry points reject this type).
    case T_BEAMBEAM4D: {
      double fx, fy;
      gauss_field(val(p.x) - q.bb.xc, val(p.y) - q.bb.yc, q.bb, &fx, &fy);
      p.px = FMA(q.bb.K, fx, p.px);
      p.py = FMA(q.bb.K, fy, p.py);
      break;
    }
    case T_SPACECHARGE: {  // values only, like the beam-beam lens
      double fx, fy;
      gauss_field(val(p.x) - q.bb.xc, val(p.y) - q.bb.yc, q.bb, &fx, &fy);
      const double zt = val(p.zeta);
      const double g = (q.sc_i2sz2 > 0.0) ? exp_cw(-((zt * zt) * q.sc_i2sz2)) : 1.0;
      const double Kg = q.bb.K * g;
      p.px = FMA(Kg, fx, p.px);
      p.py = FMA(Kg, fy, p.py);
      break;
    }
    // Rectangular aperture: lost unless xmin <= x <= xmax and ymin <= y <= ymax
    // (the boundary survives); a non-finite x or y is lost with state -1.
    case T_APERTURE_RECT: {
      const double x = val(p.x), y = val(p.y);
      if (!(x >= q.xmin && x <= q.xmax && y >= q.ymin && y <= q.ymax)) {
        bool fin = std::isfinite(x) && std::isfinite(y);
        mark_lost(p, fin ? 0 : -1, turn, elem);
      }
      break;
    }
    // Elliptic aperture with semi-axes a, b: lost if (x/a)^2 + (y/b)^2 > 1,
    // evaluated as x^2 (1/a^2) + y^2 (1/b^2).
    case T_APERTURE_ELLIPSE: {
      const double x = val(p.x), y = val(p.y);
      const double t = std::fma(x * x, q.ia2, (y * y) * q.ib2);
      if (!(t <= 1.0)) {
        bool fin = std::isfinite(x) && std::isfinite(y);
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
// Thick quadrupole: the exact flow over L of the expanded Hamiltonian
// H = pzeta - (1+delta) + (px^2 + py^2) / (2 (1+delta)) + k1 (x^2 - y^2) / 2
// (the paraxial form of the drift's square root plus the quadrupole field;
// section "Lattice modelling and single particle tracking" names thick
// quadrupoles).  Transverse motion is harmonic with w^2 = |k1| / (1+delta):
// cos/sin in the focusing plane, cosh/sinh in the other; zeta gains
// dzeta/ds = 1 - (1/rvv)(1 + (px^2 + py^2) / (2 (1+delta)^2)) integrated in
// closed form.  cos a, sin(a)/a, cosh a and sinh(a)/a at a = w |L| are the
// oscillator functions (osc_funcs) at z = |k1| L^2 / (1+delta) and -z; the
// sign of L is carried through, so that the same map with -L is its inverse.
template <class T>
static inline void osc_funcs(const T& z, T* C, T* S, T* S2, T* S3);
template <class T>
static inline void thick_quad(Part<T>& p, double k1, double L) {
  if (L == 0.0) return;
  const T aK = (k1 >= 0.0) ? k1 * p.rpp : (-k1) * p.rpp;  // |k1| / (1+delta)
  const T z = aK * (L * L);
  T C, Sa, Ch, Sha, u2, u3;
  osc_funcs(z, &C, &Sa, &u2, &u3);     // cos a, sin(a)/a
  osc_funcs(-z, &Ch, &Sha, &u2, &u3);  // cosh a, sinh(a)/a
  T* u = (k1 >= 0.0) ? &p.x : &p.y;   // focusing plane
  T* pu = (k1 >= 0.0) ? &p.px : &p.py;
  T* v = (k1 >= 0.0) ? &p.y : &p.x;
  T* pv = (k1 >= 0.0) ? &p.py : &p.px;
  const T u0 = *u, pu0 = *pu, v0 = *v, pv0 = *pv;
  const T g = (aK * L) * Sa;    // w sin(w L)
  const T gh = (aK * L) * Sha;  // w sinh(w L)
  *u = FMA(C, u0, ((L * Sa) * p.rpp) * pu0);
  *pu = FMA(-(g * p.opd), u0, C * pu0);
  *v = FMA(Ch, v0, ((L * Sha) * p.rpp) * pv0);
  *pv = FMA(gh * p.opd, v0, Ch * pv0);
  // I = integral over the element of px^2 + py^2
  const T o2 = p.opd * p.opd;
  const T A2 = pu0 * pu0, B2 = (aK * o2) * (u0 * u0);
  const T Ah2 = pv0 * pv0, Bh2 = (aK * o2) * (v0 * v0);
  const double hL = 0.5 * L;
  T I = hL * (A2 + B2);
  I = FMA(hL * (Sa * C), A2 - B2, I);
  I = FMA(-((p.opd * L) * (Sa * g)), pu0 * u0, I);
  I = FMA(mkv<T>(hL), Ah2 - Bh2, I);
  I = FMA(hL * (Sha * Ch), Ah2 + Bh2, I);
  I = FMA((p.opd * L) * (Sha * gh), pv0 * v0, I);
  // L (1 - 1/rvv) - I / (2 rvv (1+delta)^2), with 1 - 1/rvv = (delta - beta0 ptau) / (1+delta)
  p.zeta = p.zeta + FMA(L * (p.delta - p.epm1), p.rpp, -(((0.5 * p.rv0v) * (p.rpp * p.rpp)) * I));
}

// Dipole edge, non-linear model (section "Lattice modelling and single
// particle tracking": edge effects as full non-linear maps).  A hard edge of
// the field k0 whose face makes the angle e with the normal to the reference
// orbit; to first order in the field gradient the fields that Maxwell's
// equations attach to the edge (B_s = y dB_y/ds, B_x = -tan(e) y dB_y/ds)
// kick the particle by py -= k0 y T with T = tan(e + s atan(px/pz)) (s = +1
// at the entrance, -1 at the exit: the angle between the trajectory and the
// face normal), and the field missing from (or added to) the wedge between
// the face and the normal plane gives px += k0 tan(e) x.  The map is the
// canonical transformation of the generating function
//   x X' + y Y' + zeta Z' + (k0/2) y^2 T(px, py', delta) - (k0/2) tan(e) x^2
// (fringe part: py' = py - k0 y T(px, py') solved by three fixed-point
// steps; then x, y, zeta shifted by (k0/2) y^2 dT/d(px, py, pzeta)), with
//   dT/dpx = s (1 + t^2)(pz^2 + px^2) / (pz D^2),  dT/dpy = s (1 + t^2) px py / (pz D^2),
//   dT/ddelta = -s (1 + t^2) px (1+delta) / (pz D^2),  D = pz - s t px,  t = tan(e),
// and the wedge kick after it at the entrance, before it at the exit.  The
// finite extent of the fringe (fint, hgap) enters as in the linear model: a
// further py += (h tan(e) - h tan(e - psi)) y, so that the linearisation at
// the origin is the linear edge.  Lost with code -2 if pz is not real.
template <class T>
static inline void edge_nonlinear(Part<T>& p, double k0, double t, double sgn, double r21, double corr,
                                  int turn, int elem) {
  if (sgn < 0.0) p.px = FMA(r21, p.x, p.px);
  const T px = p.px, y = p.y, py = p.py;
  const T base = FMA(-px, px, p.dm1);  // (1+delta)^2 - 1 - px^2
  if (!(val(FMA(-py, py, base)) > -1.0)) { mark_lost(p, -2, turn, elem); return; }
  const T ky = k0 * y;
  const double st = sgn * t;
  T pyn = py;
  for (int k = 0; k < 3; k++) {
    const T pz = SQRT(1.0 + FMA(-pyn, pyn, base));
    const T Tv = FMA(t, pz, sgn * px) / FMA(-st, px, pz);
    pyn = FMA(-ky, Tv, py);
  }
  const T u = FMA(-pyn, pyn, base);
  if (!(val(u) > -1.0)) { mark_lost(p, -2, turn, elem); return; }
  const T pz = SQRT(1.0 + u);
  const T D = FMA(-st, px, pz);
  const T c = (sgn * (1.0 + t * t)) / (pz * (D * D));
  const T g = ((0.5 * k0) * (y * y)) * c;
  p.x = FMA(g, FMA(pz, pz, px * px), p.x);
  p.y = FMA(g, px * pyn, p.y);
  p.zeta = FMA(-(g * (px * p.opd)), p.rv0v, p.zeta);
  p.py = FMA(corr, p.y, pyn);
  if (sgn > 0.0) p.px = FMA(r21, p.x, p.px);
}

// Entire functions of z (either sign) with a = sqrt|z|: C = cos a,
// S = sin(a)/a, S2 = (1 - C)/z, S3 = (1 - S)/z for z > 0 (cosh and sinh for
// z < 0).  Series in z below |z| = 1 (each to z^9: truncation below 1e-21),
// else from sin_cw/cos_cw or two exponentials.
template <class T>
static inline void osc_funcs(const T& z, T* C, T* S, T* S2, T* S3) {
  const std::vector<double>& f = inv_fact();
  if (std::fabs(val(z)) < 1.0) {
    const T mz = -z;
    T c = mkv<T>(f[18]), s = mkv<T>(f[19]), s2 = mkv<T>(f[20]), s3 = mkv<T>(f[21]);
    for (int n = 8; n >= 0; n--) {
      c = FMA(c, mz, mkv<T>(f[2 * n]));
      s = FMA(s, mz, mkv<T>(f[2 * n + 1]));
      s2 = FMA(s2, mz, mkv<T>(f[2 * n + 2]));
      s3 = FMA(s3, mz, mkv<T>(f[2 * n + 3]));
    }
    *C = c; *S = s; *S2 = s2; *S3 = s3;
    return;
  }
  if (val(z) > 0.0) {
    const T a = SQRT(z);
    *C = COS(a);
    *S = SIN(a) / a;
  } else {
    const T a = SQRT(-z);
    const T e = EXPC(a), ei = EXPC(-a);
    *C = 0.5 * (e + ei);
    *S = (0.5 * (e - ei)) / a;
  }
  *S2 = (1.0 - *C) / z;
  *S3 = (1.0 - *S) / z;
}

// asin(v)/v = sum_n a_n v^(2n), a_n = (2n)! / (4^n n!^2 (2n+1)), n = 0..13
// (a running product t_n = t_(n-1) (2n-1) / (2n), then a_n = t_n / (2n+1)).
static const std::vector<double>& asin_coef() {
  static std::vector<double> c = [] {
    std::vector<double> v(14);
    double t = 1.0;
    for (int n = 0; n < 14; n++) {
      if (n > 0) t = (t * (double)(2 * n - 1)) / (double)(2 * n);
      v[n] = t / (double)(2 * n + 1);
    }
    return v;
  }();
  return c;
}

// asin(u)/u for |u| <= 1: the angle is halved, asin u = 2 asin v with
// v = u / sqrt(2 (1 + sqrt(1 - u^2))), until |v| < 1/4 (at most three times),
// then the series (truncation below 3e-18 there).
template <class T>
static inline T asin_over(const T& u) {
  const std::vector<double>& a = asin_coef();
  T v = u;
  double m = 1.0;
  for (int k = 0; k < 4 && std::fabs(val(v)) >= 0.25; k++) {
    v = v / SQRT(2.0 * (1.0 + SQRT(1.0 - v * v)));
    m = m + m;
  }
  const T z = v * v;
  T s = mkv<T>(a[13]);
  for (int n = 12; n >= 0; n--) s = FMA(s, z, mkv<T>(a[n]));
  if (m == 1.0) return s;
  return (m * (v / u)) * s;
}

// Thick bend, expanded model (section "Lattice modelling and single particle
// tracking": the model for large machines and small bending angles): the
// exact flow of
//   (px^2 + py^2) / (2 (1+delta)) - h x (1+delta) + k0 (x + h x^2 / 2) + k1 (x^2 - y^2) / 2,
// the Hamiltonian in the frame of curvature h with its square root expanded
// to second order in px, py and the factor (1 + h x) kept on the leading term
// only.  x is a driven oscillator, px' = F - Kx x with F = h (1+delta) - k0
// and Kx = k0 h + k1; y has py' = k1 y; and
//   zeta' = 1 - (1/rvv) (1 + h x + (px^2 + py^2) / (2 (1+delta)^2)),
// integrated in closed form with the functions of osc_funcs at
// z = K L^2 / (1+delta).  The sign of L is carried through (-L inverts).
template <class T>
static inline void bend_expanded(Part<T>& p, double k0, double h, double L, double k1) {
  const double Kx = k0 * h + k1, L2 = L * L;
  const T zx = (Kx * p.rpp) * L2;
  const T zy = ((-k1) * p.rpp) * L2;
  T C, S, S2, S3, Cy, Sy, S2y, S3y;
  osc_funcs(zx, &C, &S, &S2, &S3);
  osc_funcs(zy, &Cy, &Sy, &S2y, &S3y);
  const T x0 = p.x, px0 = p.px, y0 = p.y, py0 = p.py;
  const T F = FMA(h, p.delta, mkv<T>(h - k0));  // h (1+delta) - k0
  const T G = FMA(-Kx, x0, F);                   // px' at the entrance
  const T Gy = k1 * y0;
  const T Lr = L * p.rpp;
  p.x = FMA(C, x0, FMA(Lr * S, px0, ((L * Lr) * S2) * F));
  p.px = FMA(C, px0, (L * S) * G);
  p.y = FMA(Cy, y0, (Lr * Sy) * py0);
  p.py = FMA(Cy, py0, (L * Sy) * Gy);
  // integrals over the body of x and of px^2 + py^2, with px(s) = px0 c(s) + G s1(s):
  // int c^2 = (L/2)(1 + C S), int c s1 = (L S)^2 / 2, int s1^2 = (L^3/2)(1 - C S)/z
  // and (1 - C S)/z = S3 + S S2
  const T Ix = FMA(L * S, x0, FMA((L * Lr) * S2, px0, ((L2 * Lr) * S3) * F));
  const double hL = 0.5 * L, hL3 = 0.5 * (L2 * L);
  T I = (hL * FMA(C, S, mkv<T>(1.0))) * (px0 * px0);
  I = FMA(L2 * (S * S), px0 * G, I);
  I = FMA(hL3 * FMA(S, S2, S3), G * G, I);
  I = FMA(hL * FMA(Cy, Sy, mkv<T>(1.0)), py0 * py0, I);
  I = FMA(L2 * (Sy * Sy), py0 * Gy, I);
  I = FMA(hL3 * FMA(Sy, S2y, S3y), Gy * Gy, I);
  // L (1 - 1/rvv) = L (delta - beta0 ptau) / (1+delta)
  p.zeta = p.zeta + FMA(L * (p.delta - p.epm1), p.rpp, -(p.rv0v * FMA(h, Ix, (0.5 * (p.rpp * p.rpp)) * I)));
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
static inline void bend_full(Part<T>& p, double k0, double h, double L, int turn, int elem) {
  const double th = h * L, L2 = L * L;
  double C, S, S2, S3;
  osc_funcs(th * th, &C, &S, &S2, &S3);
  const double sn = th * S, Sh = L * S, Ch = (h * L2) * S2, D2 = 2.0 * (L2 * S2);
  const T u = FMA(-p.px, p.px, FMA(-p.py, p.py, p.dm1));  // pz^2 - 1
  if (!(val(u) > -1.0 && val(u) < INFINITY)) { mark_lost(p, -2, turn, elem); return; }
  const T pz = SQRT(1.0 + u);
  const T ph2 = 1.0 + FMA(-p.py, p.py, p.dm1);
  const T B = FMA(p.px, C, pz * sn);
  const T Q = FMA(pz, C, -(p.px * sn));
  const T r0s = FMA(p.x, sn, Sh);          // (1/h + x) sin(theta)
  const T A = FMA(-k0, r0s, B);            // px at the exit plane
  const T pzf2 = FMA(-A, A, ph2);
  if (!(val(pzf2) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
  const T pzf = SQRT(pzf2);
  const T den = pzf + Q;
  if (!(val(den) > 0.0)) { mark_lost(p, -2, turn, elem); return; }
  const T xf = FMA(p.x, C, mkv<T>(-Ch)) + r0s * ((A + B) / den);
  const T dxf = xf - p.x;
  const T chord = SQRT(FMA(dxf, dxf, (FMA(h, p.x, mkv<T>(1.0)) * FMA(h, xf, mkv<T>(1.0))) * D2));
  const T ph = SQRT(ph2);
  const T uu = (k0 * chord) / (ph + ph);
  if (!(std::fabs(val(uu)) <= 1.0)) { mark_lost(p, -2, turn, elem); return; }
  const T lh = ((L >= 0.0) ? chord : -chord) * asin_over(uu);
  const T lr = lh / ph;
  p.x = xf;
  p.px = A;
  p.y = FMA(p.py, lr, p.y);
  p.zeta = p.zeta + FMA(-p.ep, lr, mkv<T>(L));
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
    const double ax = std::fma(w, B[2 * k] - A[2 * k], A[2 * k]);
    const double ay = std::fma(w, B[2 * k + 1] - A[2 * k + 1], A[2 * k + 1]);
    const double bx = std::fma(w, B[2 * k2] - A[2 * k2], A[2 * k2]);
    const double by = std::fma(w, B[2 * k2 + 1] - A[2 * k2 + 1], A[2 * k2 + 1]);
    if ((ay > y) != (by > y)) {
      const double xi = ax + (y - ay) * (bx - ax) / (by - ay);
      if (x < xi) in = !in;
    }
  }
  return in;
}

// Inverse of one row's map (radiation off).  Returns false if the row has
// no inverse here (linear map) or the backward drift is not defined.
static bool inverse_row(Part<double>& p, const Prep& q, const RefConst& rc) {
  switch (q.type) {
    case T_DRIFT:
      drift(p, -q.L, 0, 0);
      return p.state == 1;
    case T_MULTIPOLE: {
      // the kick leaves x, y unchanged: recompute the field and take it back
      double br = q.m.c[q.m.N], bi = q.m.s[q.m.N];
      for (int n = q.m.N - 1; n >= 0; n--) {
        const double nr = std::fma(br, p.x, std::fma(-bi, p.y, q.m.c[n]));
        const double ni = std::fma(br, p.y, std::fma(bi, p.x, q.m.s[n]));
        br = nr;
        bi = ni;
      }
      p.px = p.px + br;
      p.py = p.py - bi;
      if (q.m.hxl != 0.0) {
        p.px = std::fma(-q.m.hxl, p.opd, p.px);
        p.px = std::fma(q.m.k0h, p.x, p.px);
        p.zeta = std::fma(q.m.hxl * p.rv0v, p.x, p.zeta);
      }
      return true;
    }
    case T_CAVITY: {
      const double phi = std::fma(-q.krf, p.zeta, q.lagr);
      p.ptau = std::fma(-q.qv, SIN(phi), p.ptau);
      energy_update(p, rc);
      return true;
    }
    case T_DIPEDGE:
      if (q.enl) return false;  // no inverse formed for the non-linear edge
      p.px = std::fma(-q.r21, p.x, p.px);
      p.py = std::fma(-q.r43, p.y, p.py);
      return true;
    case T_LINEARMAP: return false;
    case T_QUAD: thick_quad(p, q.k1, -q.Lq); return true;
    case T_BEND:
      if (q.bfull) bend_full(p, q.bk0, q.bh, -q.bL, 0, 0);
      else bend_expanded(p, q.bk0, q.bh, -q.bL, q.bk1);
      return p.state == 1;
    case T_BEAMBEAM4D: {  // x, y unchanged by the kick: take the same kick back
      double fx, fy;
      gauss_field(p.x - q.bb.xc, p.y - q.bb.yc, q.bb, &fx, &fy);
      p.px = std::fma(-q.bb.K, fx, p.px);
      p.py = std::fma(-q.bb.K, fy, p.py);
      return true;
    }
    case T_SPACECHARGE: {  // x, y, zeta unchanged by the kick: take the same kick back
      double fx, fy;
      gauss_field(p.x - q.bb.xc, p.y - q.bb.yc, q.bb, &fx, &fy);
      const double g = (q.sc_i2sz2 > 0.0) ? exp_cw(-((p.zeta * p.zeta) * q.sc_i2sz2)) : 1.0;
      const double Kg = q.bb.K * g;
      p.px = std::fma(-Kg, fx, p.px);
      p.py = std::fma(-Kg, fy, p.py);
      return true;
    }
    case T_XYSHIFT:
      p.x = p.x + q.dx;
      p.y = p.y + q.dy;
      return true;
    case T_SROTATION: {
      const double x = p.x, y = p.y, px = p.px, py = p.py;
      p.x = std::fma(q.cs, x, -(q.sn * y));
      p.y = std::fma(q.cs, y, q.sn * x);
      p.px = std::fma(q.cs, px, -(q.sn * py));
      p.py = std::fma(q.cs, py, q.sn * px);
      return true;
    }
    default: return true;  // markers, apertures
  }
}
}  // namespace xo

using namespace xo;

extern "C" {

// A table row the oracle accepts: a known type, a multipole order 0..10, a
// bend model 0 (expanded) or 1 (full, without gradient).
static bool row_ok(const Element& e) {
  if (e.type < 0 || e.type > T_SPACECHARGE) return false;
  if (e.type == T_MULTIPOLE && (e.order < 0 || e.order > 10)) return false;
  if (e.type == T_BEND && !(e.p[4] == 0.0 || (e.p[4] == 1.0 && e.p[3] == 0.0))) return false;
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
    derive(p, rc);
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
    derive(p, rc);
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
      // thick maps are flows: their steps compose to the same map as one pass)
      const int ty = prep[j].type;
      const double L = row_length(el[j]);
      if ((ty == T_DRIFT || ty == T_QUAD || ty == T_BEND) && L > 0.0) {
        const int64_t ns = (int64_t)std::ceil(L / ds);
        const double h = L / (double)ns;
        const double c = std::cos(fr[j].th), sn = std::sin(fr[j].th);
        for (int64_t k = 1; k <= ns; k++) {
          if (ty == T_QUAD) thick_quad(p, prep[j].k1, h);
          else if (ty == T_BEND && prep[j].bfull) bend_full(p, prep[j].bk0, prep[j].bh, h, 0, 0);
          else if (ty == T_BEND) bend_expanded(p, prep[j].bk0, prep[j].bh, h, prep[j].bk1);
          else drift(p, h, 0, 0);
          const double at = std::fma((double)k, h, pos);
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
double xo_sin(double x) { return sin_cw(x); }

// The special functions of the beam-beam kick, element-wise (for their pins).
void xo_exp(const double* x, double* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = exp_cw(x[i]);
}
void xo_one_minus_exp(const double* u, double* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = one_minus_exp(u[i]);
}
void xo_faddeeva(const double* x, const double* y, double* wr, double* wi, int64_t n) {
  for (int64_t i = 0; i < n; i++) faddeeva(x[i], y[i], &wr[i], &wi[i]);
}
// Field shape of a unit bi-Gaussian line charge (sigma_x, sigma_y) at (x, y).
void xo_gauss_field(double sx, double sy, const double* x, const double* y, double* fx, double* fy, int64_t n) {
  Element e;
  std::memset(&e, 0, sizeof(e));
  e.type = T_BEAMBEAM4D;
  e.p[0] = 1.0; e.p[1] = 1.0; e.p[2] = sx; e.p[3] = sy;
  const Reference r = {938.27208816e6, 1.0, 450e9};
  const Prep q = prepare(e, ref_const(r));
  for (int64_t i = 0; i < n; i++) gauss_field(x[i], y[i], q.bb, &fx[i], &fy[i]);
}

// The drift's (1+u)^(-1/2) - 1, element-wise (for its pins).
void xo_inv_pz_m1(const double* u, double* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = inv_pz_m1<double>(u[i]);
}
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

}  // extern "C"
