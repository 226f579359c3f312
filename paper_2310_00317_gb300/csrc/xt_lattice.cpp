// Host-side lattice compiler: the user's flat table -> device record stream.
// Compiled with -ffp-contract=off: every host constant is one IEEE operation
// sequence, so the kernel's results are reproducible bit for bit.
#include <cmath>
#include <cstring>
#include <vector>

#include "xt_internal.h"

namespace xt {

// CODATA 2018
static const double CLIGHT = 299792458.0;
static const double ME_EV = 0.51099895000e6;
static const double RE_M = 2.8179403262e-15;
static const double ALPHA = 7.2973525693e-3;
static const double HBARC_EVM = 197.3269804e-9;
static const double PI_D = 3.14159265358979323846;

Refc ref_constants(const xt_reference& r) {
  Refc c;
  c.m0 = r.mass0;
  c.q0 = r.q0;
  c.p0c = r.p0c;
  c.E0 = std::sqrt(r.p0c * r.p0c + r.mass0 * r.mass0);
  c.beta0 = r.p0c / c.E0;
  c.gamma0 = c.E0 / r.mass0;
  c.bg0 = r.p0c / r.mass0;
  c.ib0 = c.E0 / r.p0c;
  c.twoib0 = 2.0 * c.ib0;
  c.ig02 = (r.mass0 / c.E0) * (r.mass0 / c.E0);
  // classical radius of the tracked species, r_c = q^2 r_e m_e / m
  const double rc = r.q0 * r.q0 * RE_M * ME_EV / r.mass0;
  c.crad = 2.0 * rc * r.mass0 / (3.0 * r.p0c);
  c.kq = 5.0 * ALPHA * r.q0 * r.q0 / (2.0 * std::sqrt(3.0));
  c.uc15 = 1.5 * HBARC_EVM;
  return c;
}

int64_t flops_of_row(const xt_element& e, int rad_mode) {
  switch (e.type) {
    case XT_DRIFT: return 14;
    case XT_MULTIPOLE: {
      int64_t f = 8 * (int64_t)e.order + 2;
      if (e.p[22] != 0.0) f += 7;
      if (rad_mode != XT_RAD_OFF && e.p[23] > 0.0) f += (rad_mode == XT_RAD_MEAN) ? 33 : 34;
      return f;
    }
    case XT_CAVITY: return 18;
    // non-linear: three fixed-point steps (8 each), the shifts and kicks (26)
    case XT_DIPEDGE: return (e.p[4] == 2.0) ? 120 : (e.p[4] != 0.0) ? 50 : 4;  // exact wedge: two changes of plane
    case XT_LINEARMAP: return 85;
    case XT_APERTURE: return 3;
    case XT_XYSHIFT: return 2;
    case XT_SROTATION: return 12;
    case XT_APERTURE_RECT: return 0;
    case XT_APERTURE_ELLIPSE: return 5;
    // |k1|/(1+delta), a, cos, sin(a)/a, cosh and sinh(a)/a (13); the 4x4 map (18);
    // the path-length integral (36) and zeta (9)
    case XT_QUAD: return (e.p[1] == 0.0) ? 0 : 76;
    // expanded: two sets of oscillator functions (20), the 4x4 map (18), the
    // integrals (50) and zeta (10); full (the sector functions are per-element
    // constants): pz and the exit momentum (20), x (10), the chord and the arc
    // length (45), y and zeta (8)
    case XT_BEND: {
      if (e.p[4] == 0.0) return 98;
      if (e.p[3] == 0.0) return 83;
      const int64_t n = e.p[5] >= 1.0 ? (int64_t)e.p[5] : 1;
      return 83 * (n + 1) + 4 * n;  // n + 1 bodies and n thin quadrupole kicks
    }
    case XT_BEAMBEAM4D: {
      // round: the field and the kick; else two 40-term w(z) (~300 each), e^x and the rest
      const double sx2 = e.p[2] * e.p[2], sy2 = e.p[3] * e.p[3];
      return (std::fabs(sx2 - sy2) <= 1e-10 * (sx2 + sy2)) ? 20 : 650;
    }
    case XT_SPACECHARGE: {  // the same field, plus the longitudinal profile of a bunch (5)
      const double sx2 = e.p[2] * e.p[2], sy2 = e.p[3] * e.p[3];
      return ((std::fabs(sx2 - sy2) <= 1e-10 * (sx2 + sy2)) ? 20 : 650) + ((e.p[1] > 0.0) ? 5 : 0);
    }
    default: return 0;
  }
}

// Field-shape constants of a bi-Gaussian line charge into prm[3..11]: [3]
// mode (0 round when the squares agree to 1e-10, 1 sigma_x > sigma_y, 2
// otherwise), then 1/(2 s1^2), 1/(2 s2^2), s2/s1, s1/s2, 1/S, sqrt(pi)/S,
// 1/(s1 (s1 + s2)), 1/(s2 (s1 + s2)) with s1 the larger sigma and
// S = sqrt(2 (s1^2 - s2^2)); round: [4] = 1/(sigma_x^2 + sigma_y^2).
static void gauss_shape(double* prm, double sx, double sy) {
  const double sx2 = sx * sx, sy2 = sy * sy;
  if (std::fabs(sx2 - sy2) <= 1e-10 * (sx2 + sy2)) {
    prm[3] = 0.0;
    prm[4] = 1.0 / (sx2 + sy2);
    return;
  }
  const bool flat = sx2 > sy2;
  const double s1 = flat ? sx : sy, s2 = flat ? sy : sx;
  const double S = std::sqrt(2.0 * (s1 * s1 - s2 * s2));
  prm[3] = flat ? 1.0 : 2.0;
  prm[4] = 1.0 / (2.0 * (s1 * s1));
  prm[5] = 1.0 / (2.0 * (s2 * s2));
  prm[6] = s2 / s1;
  prm[7] = s1 / s2;
  prm[8] = 1.0 / S;
  prm[9] = 1.772453850905516 / S;
  prm[10] = 1.0 / (s1 * (s1 + s2));
  prm[11] = 1.0 / (s2 * (s1 + s2));
}

// The device's sine/cosine (trig_cw: Cody-Waite reduction by pi/2, Taylor
// series on |r| <= pi/4 with the coefficients of sin_table), on the host, for
// per-element constants that the device would otherwise recompute for every
// particle.  shift 0: sine, 1: cosine.
static double host_trig_cw(double x, const SinTab& t, int shift) {
  const double P1 = 1.5707963267948965579989817342720925807952880859375;
  const double P2 = 6.123233995736766035868820147291818682e-17;
  const double P3 = -1.4973849048591698329435081771059e-33;
  const double TOP = 0.63661977236758134307553505349005744813783858296183;
  const double SH = 6755399441055744.0;
  const double k = (x * TOP + SH) - SH;
  double r = std::fma(-k, P1, x);
  r = std::fma(-k, P2, r);
  r = std::fma(-k, P3, r);
  const int q = (int)(((long long)k + shift) & 3);
  const double z = r * r;
  double res;
  if (q & 1) {
    double pc = t.c[10];
    for (int i = 9; i >= 0; i--) pc = std::fma(pc, z, t.c[i]);
    res = pc;
  } else {
    double ps = t.s[9];
    for (int i = 8; i >= 1; i--) ps = std::fma(ps, z, t.s[i]);
    res = std::fma(r * z, ps, r);
  }
  return (q & 2) ? -res : res;
}

// C = cos a, S = sin(a)/a, S2 = (1 - C)/z at z = a^2 >= 0, by the device's
// oscillator-function steps (series in z below 1 with 1/n! from the special
// table, else host_trig_cw): the full bend's sector constants at z = (h L)^2.
static void sector_funcs(double z, double* C, double* S, double* S2) {
  double f[22];
  double fact = 1.0;
  for (int n = 0; n <= 21; n++) {
    if (n > 0) fact = fact * (double)n;
    f[n] = 1.0 / fact;
  }
  if (std::fabs(z) < 1.0) {
    const double mz = -z;
    double c = f[18], s = f[19], s2 = f[20];
    for (int n = 8; n >= 0; n--) {
      c = std::fma(c, mz, f[2 * n]);
      s = std::fma(s, mz, f[2 * n + 1]);
      s2 = std::fma(s2, mz, f[2 * n + 2]);
    }
    *C = c; *S = s; *S2 = s2;
    return;
  }
  const SinTab t = sin_table();
  const double a = std::sqrt(z);
  *C = host_trig_cw(a, t, 1);
  *S = host_trig_cw(a, t, 0) / a;
  *S2 = (1.0 - *C) / z;
}

static void put(std::vector<uint8_t>& b, const void* p, size_t n) {
  const uint8_t* s = (const uint8_t*)p;
  b.insert(b.end(), s, s + n);
}

int compile_lattice(const xt_element* table, int64_t n, const Refc& rc, Lattice* out,
                    std::string* err) {
  out->bytes.clear();
  out->rec_off.clear();
  out->row_rec.assign((size_t)n, -1);
  out->thick = false;
  out->rec_bytes.clear();
  out->flops.assign((size_t)n, 0);
  out->n_el = n;
  for (int64_t i = 0; i < n; i++) {
    const xt_element& e = table[i];
    std::vector<double> prm;
    uint16_t flags = 0;
    switch (e.type) {
      case XT_MARKER: continue;
      case XT_DRIFT: prm = {e.p[0]}; break;
      case XT_MULTIPOLE: {
        if (e.order < 0 || e.order > XT_MAX_ORDER) {
          *err = "element " + std::to_string(i) + ": multipole order outside 0..10";
          return XT_ERR_UNSUPPORTED;
        }
        const double hxl = e.p[22], lrad = e.p[23];
        if (!(lrad >= 0.0)) {
          *err = "element " + std::to_string(i) + ": L_rad must be >= 0";
          return XT_ERR_INVALID;
        }
        prm.assign(MP_COEF + 2 * (e.order + 1), 0.0);
        prm[MP_HXL] = hxl;
        prm[MP_K0H] = (lrad > 0.0) ? (e.p[0] * hxl) / lrad : 0.0;
        prm[MP_CRL] = rc.crad * lrad;
        prm[MP_ILR2] = (lrad > 0.0) ? 1.0 / (lrad * lrad) : 0.0;
        prm[MP_KQL] = rc.kq * lrad;
        prm[MP_LRAD] = lrad;
        double fact = 1.0;
        for (int k = 0; k <= e.order; k++) {
          if (k > 0) fact = fact * (double)k;
          prm[MP_COEF + 2 * k] = e.p[k] / fact;
          prm[MP_COEF + 2 * k + 1] = e.p[11 + k] / fact;
        }
        if (hxl != 0.0) flags |= REC_CURV;
        if (lrad > 0.0) flags |= REC_RAD;
        if (e.p[0] == 0.0 && e.p[11] == 0.0 && hxl == 0.0) flags |= REC_PURE;
        if (hxl != 0.0 && hxl == e.p[0] && e.p[11] == 0.0) flags |= REC_BEND;
        break;
      }
      case XT_CAVITY: {
        const double V = e.p[0], f = e.p[1], lag = e.p[2];
        prm = {(2.0 * PI_D * f) / (rc.beta0 * CLIGHT), lag * PI_D / 180.0, (rc.q0 * V) / rc.p0c};
        break;
      }
      case XT_DIPEDGE: {
        const double h = e.p[0], e1 = e.p[1], hgap = e.p[2], fint = e.p[3];
        if (!((e.p[4] == 0.0 || e.p[4] == 1.0 || e.p[4] == 2.0) && (e.p[5] == 0.0 || e.p[5] == 1.0))) {
          *err = "element " + std::to_string(i) + ": dipole edge model must be 0, 1 or 2 and face 0 or 1";
          return XT_ERR_INVALID;
        }
        const double psi = 2.0 * h * hgap * fint * (1.0 + std::sin(e1) * std::sin(e1)) / std::cos(e1);
        const double r21 = h * std::tan(e1), r43 = -h * std::tan(e1 - psi);
        if (e.p[4] == 2.0) {  // exact wedge: no wedge kick, r43, k0, t = 0 on the face, s, correction, cos, sin
          prm = {0.0, r43, h, 0.0, (e.p[5] != 0.0) ? -1.0 : 1.0, r21 + r43, std::cos(e1), std::sin(e1)};
          flags |= REC_ENL | REC_EWEDGE;
        } else if (e.p[4] == 1.0) {  // non-linear: r21, r43, k0, tan(e1), +1 entrance / -1 exit, correction
          prm = {r21, r43, h, std::tan(e1), (e.p[5] != 0.0) ? -1.0 : 1.0, r21 + r43};
          flags |= REC_ENL;
        } else {
          prm = {r21, r43};
        }
        break;
      }
      case XT_LINEARMAP: {
        // (x,px,y,py,zeta,pzeta) -> (x,px,y,py,zeta,ptau): row 5 times beta0,
        // column 5 times 1/beta0, d_5 times beta0.
        prm.assign(42, 0.0);
        for (int r = 0; r < 6; r++) {
          for (int c = 0; c < 6; c++) {
            double v = e.p[6 * r + c];
            if (r == 5 && c != 5) v = v * rc.beta0;
            else if (c == 5 && r != 5) v = v * rc.ib0;
            prm[6 * r + c] = v;
          }
          prm[36 + r] = (r == 5) ? e.p[36 + r] * rc.beta0 : e.p[36 + r];
        }
        break;
      }
      case XT_APERTURE:
        prm = {e.p[0] * e.p[0], e.p[0] * (1.0 - 9.5367431640625e-07) * 0.70710678118654752};
        break;
      case XT_XYSHIFT: prm = {e.p[0], e.p[1]}; break;
      case XT_SROTATION: prm = {std::cos(e.p[0]), std::sin(e.p[0])}; break;
      case XT_APERTURE_RECT:
        if (!(e.p[0] <= e.p[1] && e.p[2] <= e.p[3])) {
          *err = "element " + std::to_string(i) + ": rectangular aperture needs x_min <= x_max, y_min <= y_max";
          return XT_ERR_INVALID;
        }
        prm = {e.p[0], e.p[1], e.p[2], e.p[3]};
        break;
      case XT_BEAMBEAM4D: {
        const double qN = e.p[0], bs = e.p[1], sx = e.p[2], sy = e.p[3];
        if (!(sx > 0.0 && sy > 0.0 && bs > 0.0 && bs <= 1.0)) {
          *err = "element " + std::to_string(i) + ": beam-beam lens needs sigma_x, sigma_y > 0 and 0 < beta_s <= 1";
          return XT_ERR_INVALID;
        }
        // kick of a counter-moving Gaussian bunch integrated over the crossing
        const double K = 2.0 * rc.q0 * qN * (RE_M * ME_EV) / rc.p0c * ((1.0 + rc.beta0 * bs) / (rc.beta0 + bs));
        prm.assign(12, 0.0);
        prm[0] = K;
        prm[1] = e.p[4];
        prm[2] = e.p[5];
        gauss_shape(prm.data(), sx, sy);
        break;
      }
      case XT_SPACECHARGE: {
        const double lam0 = e.p[0], sz = e.p[1], sx = e.p[2], sy = e.p[3], L = e.p[4];
        if (!(sx > 0.0 && sy > 0.0 && sz >= 0.0 && lam0 >= 0.0 && L >= 0.0) || !std::isfinite(lam0) ||
            !std::isfinite(L) || !std::isfinite(sz)) {
          *err = "element " + std::to_string(i) +
                 ": space-charge lens needs sigma_x, sigma_y > 0, sigma_z >= 0, a line density >= 0 and L >= 0";
          return XT_ERR_INVALID;
        }
        // the beam's own field, electric and magnetic forces cancelling to 1/gamma^2
        const double rcl = rc.q0 * rc.q0 * RE_M * ME_EV / rc.m0;
        prm.assign(13, 0.0);
        prm[0] = 2.0 * rcl * lam0 * L / (rc.beta0 * rc.beta0 * rc.gamma0 * rc.gamma0 * rc.gamma0);
        prm[1] = e.p[5];
        prm[2] = e.p[6];
        gauss_shape(prm.data(), sx, sy);
        prm[12] = (sz > 0.0) ? 1.0 / (2.0 * (sz * sz)) : 0.0;
        break;
      }
      case XT_QUAD: {
        const double k1 = e.p[0], L = e.p[1];
        if (!(L >= 0.0) || !std::isfinite(L) || !std::isfinite(k1)) {
          *err = "element " + std::to_string(i) + ": thick quadrupole needs a finite k1 and a finite length L >= 0";
          return XT_ERR_INVALID;
        }
        if (L == 0.0) continue;  // no effect
        prm = {(k1 >= 0.0) ? k1 : -k1, L};
        if (k1 >= 0.0) flags |= REC_QF;
        break;
      }
      case XT_BEND: {
        const double k0 = e.p[0], h = e.p[1], L = e.p[2], k1 = e.p[3], model = e.p[4];
        if (!std::isfinite(k0) || !std::isfinite(h) || !std::isfinite(k1) || !std::isfinite(L) || !(L >= 0.0)) {
          *err = "element " + std::to_string(i) + ": thick bend needs finite k0, h, k1 and a length L >= 0";
          return XT_ERR_INVALID;
        }
        const double nk = e.p[5];
        if (!(model == 0.0 || model == 1.0) || !(nk >= 0.0 && nk <= 64.0 && nk == std::floor(nk))) {
          *err = "element " + std::to_string(i) + ": thick bend model must be 0 (expanded) or 1 (full), "
                 "and the number of gradient kicks an integer in 0..64";
          return XT_ERR_INVALID;
        }
        prm = {k0, h, L, k1};
        if (model == 1.0) {  // the sector's constants once: C, S, S2 at z = (h L)^2
          flags |= REC_BFULL;
          const double th = h * L;
          double C, S, S2;
          sector_funcs(th * th, &C, &S, &S2);
          prm.push_back(C);
          prm.push_back(S);
          prm.push_back(S2);
          if (k1 != 0.0) {  // the gradient by n kicks between exact bodies (see bend_full_kicks)
            flags |= REC_BKICK;
            const int n = nk >= 1.0 ? (int)nk : 1;
            const double lh = L / (2.0 * n), ls = L / (double)n;
            prm.push_back((double)n);
            sector_funcs((h * lh) * (h * lh), &C, &S, &S2);
            prm.push_back(C);
            prm.push_back(S);
            prm.push_back(S2);
            sector_funcs((h * ls) * (h * ls), &C, &S, &S2);
            prm.push_back(C);
            prm.push_back(S);
            prm.push_back(S2);
            prm.push_back(lh);
            prm.push_back(ls);
            prm.push_back(k1 * ls);
          }
        }
        break;
      }
      case XT_APERTURE_ELLIPSE:
        if (!(e.p[0] > 0.0 && e.p[1] > 0.0)) {
          *err = "element " + std::to_string(i) + ": elliptic aperture needs a > 0 and b > 0";
          return XT_ERR_INVALID;
        }
        prm = {1.0 / (e.p[0] * e.p[0]), 1.0 / (e.p[1] * e.p[1])};
        break;
      default:
        *err = "element " + std::to_string(i) + ": unknown type " + std::to_string(e.type);
        return XT_ERR_UNSUPPORTED;
    }
    if (prm.size() % 2) prm.push_back(0.0);
    RecHdr h;
    std::memset(&h, 0, sizeof(h));
    h.type = (uint16_t)e.type;
    h.order = (uint16_t)(e.type == XT_MULTIPOLE ? e.order : 0);
    h.flags = flags;
    const size_t bytes = sizeof(RecHdr) + prm.size() * sizeof(double);
    h.size16 = (uint16_t)(bytes / 16);
    h.elem = (uint32_t)i;
    out->row_rec[(size_t)i] = (int32_t)out->bytes.size();
    if (e.type == XT_BEAMBEAM4D || e.type == XT_SPACECHARGE || e.type == XT_QUAD || e.type == XT_BEND ||
        (e.type == XT_DIPEDGE && (flags & REC_ENL)))
      out->thick = true;
    out->rec_off.push_back((uint32_t)out->bytes.size());
    out->rec_bytes.push_back((uint32_t)bytes);
    put(out->bytes, &h, sizeof(h));
    put(out->bytes, prm.data(), prm.size() * sizeof(double));
  }
  // FNV-1a hash of the record stream (autotune cache key)
  uint64_t hsh = 1469598103934665603ULL;
  for (uint8_t b : out->bytes) { hsh ^= b; hsh *= 1099511628211ULL; }
  out->hash = hsh ^ (uint64_t)n;
  return XT_OK;
}

void build_chunks(const Lattice& lat, uint32_t chunk_bytes, std::vector<Chunk>* out) {
  out->clear();
  Chunk c = {0, 0, 0, 0};
  for (size_t r = 0; r < lat.rec_off.size(); r++) {
    const uint32_t b = lat.rec_bytes[r];
    if (c.nrec > 0 && c.bytes + b > chunk_bytes) {
      out->push_back(c);
      c = {lat.rec_off[r], 0, 0, 0};
    }
    if (c.nrec == 0) c.off = lat.rec_off[r];
    c.bytes += b;
    c.nrec += 1;
  }
  if (c.nrec > 0) out->push_back(c);
}

SinTab sin_table() {
  SinTab t;
  double fact = 1.0;
  for (int n = 1; n <= 21; n++) {
    fact = fact * (double)n;
    const int k = n / 2;
    if (n & 1) {
      if (k < 10) t.s[k] = ((k & 1) ? -1.0 : 1.0) / fact;
    } else if (k < 11) {
      t.c[k] = ((k & 1) ? -1.0 : 1.0) / fact;
    }
  }
  t.s[0] = 1.0;
  t.c[0] = 1.0;
  return t;
}

// Constant table of the beam-beam kick: [0] L, [1..40] the coefficients of
// p(Z) in Weideman's rational expansion of the Faddeeva function
// (J. A. C. Weideman, SIAM J. Numer. Anal. 31 (1994) 1497; N = 40 terms,
// L = (N / sqrt 2)^(1/2), the cosine transform of e^(-t^2)(L^2 + t^2) at
// t = L tan(theta/2) by a plain DFT), [41..62] 1/n! for n = 0..21 (the running
// product n! rounds beyond 18!); and for the thick bend's arc length [63..76]
// the coefficients a_n of
// asin(v)/v = sum a_n v^(2n), a_n = (2n)! / (4^n n!^2 (2n+1)) from the
// running product t_n = t_(n-1) (2n-1) / (2n), a_n = t_n / (2n+1).
// [77..277] 1/k for k = 0..200 (the photon-count recurrence; entry 0 unused).
void special_table(double* out) {
  const int N = 40, M = 2 * N, M2 = 2 * M;
  const double L = std::sqrt((double)N / std::sqrt(2.0));
  std::vector<double> f(M2), fs(M2);
  f[0] = 0.0;
  for (int j = 1; j < M2; j++) {
    const int k = j - M;
    const double theta = (double)k * PI_D / (double)M;
    const double t = L * std::tan(theta / 2.0);
    f[j] = std::exp(-t * t) * (L * L + t * t);
  }
  for (int j = 0; j < M2; j++) fs[j] = f[(j + M) % M2];
  out[0] = L;
  for (int n = 0; n < N; n++) {
    const int m = n + 1;
    double acc = 0.0;
    for (int j = 0; j < M2; j++) acc = acc + fs[j] * std::cos(2.0 * PI_D * (double)((j * m) % M2) / (double)M2);
    out[1 + n] = acc / (double)M2;
  }
  double fact = 1.0;
  for (int n = 0; n <= 21; n++) {
    if (n > 0) fact = fact * (double)n;
    out[XT_SPECIAL_FACT + n] = 1.0 / fact;
  }
  double t = 1.0;
  for (int n = 0; n < 14; n++) {
    if (n > 0) t = (t * (double)(2 * n - 1)) / (double)(2 * n);
    out[XT_SPECIAL_ASIN + n] = t / (double)(2 * n + 1);
  }
  out[XT_SPECIAL_RECIP] = 0.0;
  for (int k = 1; k <= 200; k++) out[XT_SPECIAL_RECIP + k] = 1.0 / (double)k;
}

// Photon-number spectrum of synchrotron radiation in xi = u/u_c:
// dN/dxi ~ G(xi) = int_xi^inf K_{5/3}(t) dt, total 5 pi/3.  With
// K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt and the order of
// integration exchanged, the tail is S(xi) = int_xi^inf G =
// int_0^inf exp(-xi cosh t) cosh(5t/3) / cosh^2 t dt, evaluated by the
// trapezoidal rule with step 0.05 in t (the integrand is even and analytic in
// a strip about the real axis, so the rule converges geometrically) until
// xi cosh t > 60; F = 1 - S / (5 pi / 3) at 2048 knots xi = 1e-7 (4e8)^(i/2047).
// The quantum-radiation tests compare this model with an independent
// implementation of the same steps bit for bit, so the steps are fixed.
//
// Guide table (H. C. Chen, Y. Asau, Technometrics 16 (1974) 615) for the
// inverse CDF: G[j] = max{i : F[i] <= j/4096}; a uniform u starts its search
// at G[floor(4096 u)] and walks up to max{i : F[i] <= u}.
void photon_table(std::vector<double>* xi, std::vector<double>* F, std::vector<int32_t>* guide) {
  const int K = 2048, M = 4096;
  const double xmin = 1e-7, xmax = 40.0, norm = 5.0 * PI_D / 3.0, h = 0.05;
  xi->resize(K);
  F->resize(K);
  for (int i = 0; i < K; i++) {
    const double e = (double)i / (double)(K - 1);
    const double x = xmin * std::pow(xmax / xmin, e);
    double acc = 0.0;
    for (int j = 0;; j++) {
      const double t = j * h;
      const double ch = std::cosh(t);
      const double g = std::exp(-x * ch) * std::cosh(5.0 * t / 3.0) / (ch * ch);
      acc = acc + (j == 0 ? 0.5 : 1.0) * g;
      if (x * ch > 60.0 && j > 10) break;
    }
    (*xi)[i] = x;
    (*F)[i] = 1.0 - (h * acc) / norm;
  }
  guide->resize(M);
  int i = 0;
  for (int j = 0; j < M; j++) {
    const double t = (double)j / (double)M;
    while (i + 1 < K && (*F)[i + 1] <= t) i++;
    (*guide)[j] = i;
  }
  // after the K knots: 1 / (F[k+1] - F[k]) for each interval (0 for the last
  // knot), then 1 / F[0], so that the sampler multiplies instead of dividing
  F->resize(2 * K + 1);
  for (int k = 0; k + 1 < K; k++) (*F)[K + k] = 1.0 / ((*F)[k + 1] - (*F)[k]);
  (*F)[2 * K - 1] = 0.0;
  (*F)[2 * K] = 1.0 / (*F)[0];
}

}  // namespace xt
