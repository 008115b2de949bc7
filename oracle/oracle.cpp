// FP64 CPU oracle for the metadynamics-of-paths effective potential.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path is
// checked against.  It shares no code, header, table or constant generator with the CUDA
// library; only the tests, the package smoke check and the CPU-baseline leg of the
// benchmark may load it.
//
// What it computes (paper: arXiv 2501.11962, Section 1.1):
//   V_eff = U(R^1) + sum_{n=1}^{N-1} K/2 |R^{n+1} - R^n - L^n|^2           (Eq. 3)
//   K_i = m_i nu / (2 dt),  L^n_i = (dt / (m_i nu)) F^n_i,  F = -grad U        (Sec. 1.1)
//   eta^n = R^{n+1} - R^n - L^n                                            (text below Eq. 5)
// and the exact gradient, which the paper writes as the effective forces of Eqs. 5-7 with a
// finite-difference stand-in for the Hessian-vector product:
//   dV/dR^1 = -F^1 - K eta^1 + 1/2 H(R^1) eta^1
//   dV/dR^n =  K eta^{n-1} - K eta^n + 1/2 H(R^n) eta^n        (1 < n < N)
//   dV/dR^N =  K eta^{N-1}
// The paper's FD form (Eq. 5, Eq. 6, Eq. 7) is also provided, with the displacement
// eps = h / max_i |eta^n_i| (the paper gives no formula for eps; this is the reading used).
//
// Physical model (the paper's force field is not available):
//   Lennard-Jones with Lorentz-Berthelot mixing + Tironi reaction field, both with the
//   shifted-force cutoff modifier phi_sf(r) = phi(r) - phi(rc) - (r - rc) phi'(rc), r < rc;
//   harmonic bonds k/2 (d - r0)^2 and harmonic angles k/2 (theta - theta0)^2;
//   nonbonded exclusions: same molecule and |local_i - local_j| <= 2.
//
// Parity pins (tests/test_oracle_pins.py): closed forms of single pairs, O(Q^2) brute force vs
// the cell list, Newton's third law, translation invariance, central differences of U,
// complex-step and dual-number Hessian-vector products, dense-Hessian symmetry, the rotation
// identity, the U = 0 discrete-Laplacian case, complex-step derivatives of V_eff, Eqs. 5-7,
// Philox known-answer vectors, NVE energy drift.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kCoulomb = 138.935458;      // kJ mol^-1 nm e^-2
constexpr double kBoltzmann = 0.0083144626;  // kJ mol^-1 K^-1

// ---------------------------------------------------------------------------------------------
// scalar types: double, complex (complex step), Dual (forward mode)

struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return {s, a.d / (2.0 * s)}; }
inline Dual acos(Dual a) { return {std::acos(a.v), -a.d / std::sqrt(1.0 - a.v * a.v)}; }

inline double re(double a) { return a; }
inline double re(const std::complex<double>& a) { return a.real(); }
inline double re(const Dual& a) { return a.v; }
template <class T> T make(double a) { return T(a); }

using cplx = std::complex<double>;
inline cplx acos(const cplx& a) { return std::acos(a); }
inline cplx sqrt(const cplx& a) { return std::sqrt(a); }
inline Dual exp(Dual a) { const double e = std::exp(a.v); return {e, e * a.d}; }
using std::acos;
using std::sqrt;
using std::exp;

constexpr double kTwoOverSqrtPi = 1.1283791670955126;   // 2 / sqrt(pi)

// erfc(b r) for the scalar types.  Dual carries the derivative -2b/sqrt(pi) exp(-b^2 r^2) r';
// complex carries it on the imaginary part, which is exact to first order (the complex step
// uses imaginary parts of 1e-20).
inline double erfc_b(double r, double b) { return std::erfc(b * r); }
inline Dual erfc_b(const Dual& r, double b) {
  return {std::erfc(b * r.v), -kTwoOverSqrtPi * b * std::exp(-b * b * r.v * r.v) * r.d};
}
inline cplx erfc_b(const cplx& r, double b) {
  const double x = r.real();
  return {std::erfc(b * x), -kTwoOverSqrtPi * b * std::exp(-b * b * x * x) * r.imag()};
}

}  // namespace

extern "C" {

// Host description of one system; every pointer is a host array owned by the caller.
struct orc_system {
  int32_t Q;
  int32_t n_types;
  double box[3];
  const int32_t* type;
  const double* sigma;
  const double* eps;
  const double* charge;
  const double* mass;
  const int32_t* mol_id;
  const int32_t* mol_local;
  int32_t n_bonds;
  const int32_t* bond_ij;
  const double* bond_r0;
  const double* bond_k;
  int32_t n_angles;
  const int32_t* angle_ijk;
  const double* angle_th0;
  const double* angle_k;
  double rc;
  double eps_rf;
  int32_t cutoff_mode;  // 0 = shifted force, 1 = potential shift
  double dt_path;
  double nu_path;
  int32_t elec;         // 0 = reaction field, 1 = Ewald real space (erfc, with the exclusion and
                        //     self terms; the reciprocal part is computed elsewhere)
  double ew_beta;       // Ewald splitting parameter, 1/nm
};

}  // extern "C"

namespace {

struct PairParams {
  double c6, c12, qq;          // 4 eps sigma^6, 4 eps sigma^12, f q_i q_j
  double phi_rc, dphi_rc;      // potential and its r-derivative at rc
};

struct Model {
  const orc_system& s;
  bool ewald;
  double beta;
  double krf, crf;
  double rc6, rc7, rc12, rc13;     // powers of rc for the cutoff constants
  std::vector<double> c6t, c12t;   // per type pair, Lorentz-Berthelot
  explicit Model(const orc_system& sys) : s(sys), ewald(sys.elec == 1), beta(sys.ew_beta) {
    const double rc = s.rc;
    krf = (s.eps_rf - 1.0) / ((2.0 * s.eps_rf + 1.0) * rc * rc * rc);
    crf = 1.0 / rc + krf * rc * rc;
    rc6 = std::pow(rc, 6);
    rc7 = std::pow(rc, 7);
    rc12 = std::pow(rc, 12);
    rc13 = std::pow(rc, 13);
    const int nt = s.n_types;
    c6t.resize(nt * nt);
    c12t.resize(nt * nt);
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b) {
        const double sig = 0.5 * (s.sigma[a] + s.sigma[b]);     // Lorentz
        const double eps = std::sqrt(s.eps[a] * s.eps[b]);       // Berthelot
        const double s6 = std::pow(sig, 6);
        c6t[a * nt + b] = 4.0 * eps * s6;
        c12t[a * nt + b] = 4.0 * eps * s6 * s6;
      }
  }
  bool excluded(int i, int j) const {
    return s.mol_id[i] == s.mol_id[j] && std::abs(s.mol_local[i] - s.mol_local[j]) <= 2;
  }
  PairParams params(int i, int j) const {
    const int t = s.type[i] * s.n_types + s.type[j];
    PairParams p;
    p.c6 = c6t[t];
    p.c12 = c12t[t];
    p.qq = kCoulomb * s.charge[i] * s.charge[j];
    const double rc = s.rc;
    p.phi_rc = p.c12 / rc12 - p.c6 / rc6;
    p.dphi_rc = -12.0 * p.c12 / rc13 + 6.0 * p.c6 / rc7;
    if (ewald) {
      const double e = std::erfc(beta * rc), g = kTwoOverSqrtPi * beta * std::exp(-beta * beta * rc * rc);
      p.phi_rc += p.qq * e / rc;
      p.dphi_rc -= p.qq * (e / (rc * rc) + g / rc);
    } else {
      p.phi_rc += p.qq * (1.0 / rc + krf * rc * rc - crf);
      p.dphi_rc += p.qq * (-1.0 / (rc * rc) + 2.0 * krf * rc);
    }
    return p;
  }
  // Ewald exclusion correction of an excluded pair: -f q_i q_j erf(beta r) / r (its reciprocal-
  // space interaction is removed; no cutoff), value and r-derivative
  template <class T>
  void phi_excl(double qq, const T& r, T* val, T* der) const {
    T ir = make<T>(1.0) / r;
    T erf_ = make<T>(1.0) - erfc_b(r, beta);
    *val = -qq * erf_ * ir;
    *der = qq * (erf_ * ir * ir - kTwoOverSqrtPi * beta * exp(make<T>(-beta * beta) * r * r) * ir);
  }
  double phi_excl2(double qq, double r) const {
    const double ir = 1.0 / r, erf_ = std::erf(beta * r), g = kTwoOverSqrtPi * beta * std::exp(-beta * beta * r * r);
    // d2/dr2 of erf(b r)/r = 2 erf/r^3 - g (2/r^2 + 2 b^2)
    return -qq * (2.0 * erf_ * ir * ir * ir - g * (2.0 * ir * ir + 2.0 * beta * beta));
  }
  // self term of the Ewald sum, -f beta / sqrt(pi) sum_i q_i^2 (a constant)
  double self_energy() const {
    if (!ewald) return 0.0;
    double q2 = 0.0;
    for (int i = 0; i < s.Q; ++i) q2 += s.charge[i] * s.charge[i];
    return -kCoulomb * beta / std::sqrt(M_PI) * q2;
  }
  // phi(r) and phi'(r) with the cutoff modifier, for r < rc
  template <class T>
  void phi(const PairParams& p, const T& r, T* val, T* der) const {
    T ir = make<T>(1.0) / r;
    T ir2 = ir * ir;
    T ir6 = ir2 * ir2 * ir2;
    T v = p.c12 * ir6 * ir6 - p.c6 * ir6;
    T d = (-12.0 * p.c12 * ir6 * ir6 + 6.0 * p.c6 * ir6) * ir;
    if (ewald) {
      const T e = erfc_b(r, beta);
      v = v + p.qq * e * ir;
      d = d - p.qq * (e * ir2 + kTwoOverSqrtPi * beta * exp(make<T>(-beta * beta) * r * r) * ir);
    } else {
      v = v + p.qq * (ir + krf * r * r - crf);
      d = d + p.qq * (-ir2 + 2.0 * krf * r);
    }
    if (s.cutoff_mode == 0) {
      v = v - p.phi_rc - (r - s.rc) * p.dphi_rc;
      d = d - p.dphi_rc;
    } else {
      v = v - p.phi_rc;
    }
    *val = v;
    *der = d;
  }
  // second derivative phi''(r) (the modifiers are at most linear in r)
  double phi2(const PairParams& p, double r) const {
    double ir = 1.0 / r, ir2 = ir * ir, ir6 = ir2 * ir2 * ir2;
    const double lj = (156.0 * p.c12 * ir6 * ir6 - 42.0 * p.c6 * ir6) * ir2;
    if (ewald) {
      // d2/dr2 of erfc(b r)/r = 2 erfc/r^3 + g (2/r^2 + 2 b^2), g = 2b/sqrt(pi) exp(-b^2 r^2)
      const double g = kTwoOverSqrtPi * beta * std::exp(-beta * beta * r * r);
      return lj + p.qq * (2.0 * std::erfc(beta * r) * ir2 * ir + g * (2.0 * ir2 + 2.0 * beta * beta));
    }
    return lj + p.qq * (2.0 * ir2 * ir + 2.0 * krf);
  }
};

template <class T>
inline void min_image(const orc_system& s, const T* xi, const T* xj, T* d) {
  for (int k = 0; k < 3; ++k) {
    T dk = xi[k] - xj[k];
    d[k] = dk - s.box[k] * std::nearbyint(re(dk) / s.box[k]);
  }
}

// Calls fn(i, j) for every unordered pair (i < j) whose minimum-image distance (on real parts)
// is < rc.  method 0: linked cells (brute force when a box edge holds fewer than 3 cells);
// method 1: O(Q^2) brute force.
template <class Fn>
void for_each_pair(const orc_system& s, const double* x, int method, Fn&& fn) {
  const int Q = s.Q;
  const double rc2 = s.rc * s.rc;
  auto consider = [&](int i, int j) {
    double d[3];
    min_image(s, x + 3 * i, x + 3 * j, d);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < rc2) fn(i, j);
  };
  int nc[3];
  for (int k = 0; k < 3; ++k) nc[k] = (int)std::floor(s.box[k] / s.rc);
  if (method == 1 || nc[0] < 3 || nc[1] < 3 || nc[2] < 3) {
    for (int i = 0; i < Q; ++i)
      for (int j = i + 1; j < Q; ++j) consider(i, j);
    return;
  }
  const int ncell = nc[0] * nc[1] * nc[2];
  std::vector<int> head(ncell, -1), next(Q, -1), cell(Q);
  for (int i = 0; i < Q; ++i) {
    int c[3];
    for (int k = 0; k < 3; ++k) {
      double w = x[3 * i + k] - s.box[k] * std::floor(x[3 * i + k] / s.box[k]);
      c[k] = std::min((int)std::floor(w / (s.box[k] / nc[k])), nc[k] - 1);
    }
    cell[i] = (c[0] * nc[1] + c[1]) * nc[2] + c[2];
  }
  for (int i = Q - 1; i >= 0; --i) { next[i] = head[cell[i]]; head[cell[i]] = i; }
  for (int i = 0; i < Q; ++i) {
    int ci = cell[i];
    int cz = ci % nc[2], cy = (ci / nc[2]) % nc[1], cx = ci / (nc[1] * nc[2]);
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int ox = (cx + dx + nc[0]) % nc[0], oy = (cy + dy + nc[1]) % nc[1], oz = (cz + dz + nc[2]) % nc[2];
          for (int j = head[(ox * nc[1] + oy) * nc[2] + oz]; j >= 0; j = next[j])
            if (j > i) consider(i, j);
        }
  }
}

// Nonbonded (pair) part of U and F, accumulated into F and *u.
template <class T>
void nonbonded_T(const orc_system& s, const T* x, T* F, T* u, int method) {
  const Model m(s);
  std::vector<double> xr(3 * (size_t)s.Q);
  for (size_t k = 0; k < xr.size(); ++k) xr[k] = re(x[k]);
  *u += m.self_energy();
  for_each_pair(s, xr.data(), method, [&](int i, int j) {
    const bool ex = m.excluded(i, j);
    if (ex && !m.ewald) return;
    T d[3];
    min_image(s, x + 3 * i, x + 3 * j, d);
    T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    T v, dv;
    if (ex) m.phi_excl(kCoulomb * s.charge[i] * s.charge[j], r, &v, &dv);
    else m.phi(m.params(i, j), r, &v, &dv);
    *u += v;
    for (int k = 0; k < 3; ++k) {
      T f = -dv * d[k] / r;
      F[3 * i + k] += f;
      F[3 * j + k] -= f;
    }
  });
}

// Harmonic bonds k/2 (d - r0)^2.
template <class T>
void bonds_T(const orc_system& s, const T* x, T* F, T* u) {
  for (int b = 0; b < s.n_bonds; ++b) {
    int i = s.bond_ij[2 * b], j = s.bond_ij[2 * b + 1];
    T d[3];
    min_image(s, x + 3 * i, x + 3 * j, d);
    T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    T dr = r - s.bond_r0[b];
    *u += 0.5 * s.bond_k[b] * dr * dr;
    for (int k = 0; k < 3; ++k) {
      T f = -s.bond_k[b] * dr * d[k] / r;
      F[3 * i + k] += f;
      F[3 * j + k] -= f;
    }
  }
}

// Harmonic angles k/2 (theta - theta0)^2, theta the angle at vertex j between i-j and l-j.
template <class T>
void angles_T(const orc_system& s, const T* x, T* F, T* u) {
  for (int a = 0; a < s.n_angles; ++a) {
    int i = s.angle_ijk[3 * a], j = s.angle_ijk[3 * a + 1], l = s.angle_ijk[3 * a + 2];
    T p[3], q[3];
    min_image(s, x + 3 * i, x + 3 * j, p);
    min_image(s, x + 3 * l, x + 3 * j, q);
    T pp = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    T qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    T pq = p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
    T np_ = sqrt(pp), nq = sqrt(qq);
    T c = pq / (np_ * nq);
    T th = acos(c);
    T dth = th - s.angle_th0[a];
    *u += 0.5 * s.angle_k[a] * dth * dth;
    // dU/dcos = k (theta - theta0) dtheta/dcos, dtheta/dcos = -1/sin(theta)
    T sn = sqrt(make<T>(1.0) - c * c);
    T g = -s.angle_k[a] * dth / sn;
    for (int k = 0; k < 3; ++k) {
      T dcp = q[k] / (np_ * nq) - c * p[k] / pp;   // d cos / d p
      T dcq = p[k] / (np_ * nq) - c * q[k] / qq;   // d cos / d q
      T fi = -g * dcp, fl = -g * dcq;
      F[3 * i + k] += fi;
      F[3 * l + k] += fl;
      F[3 * j + k] -= fi + fl;
    }
  }
}

// U and F = -grad U at positions x (T = double, complex or Dual; decisions on real parts).
template <class T>
void forces_T(const orc_system& s, const T* x, T* F, T* U, int method) {
  for (size_t k = 0; k < 3 * (size_t)s.Q; ++k) F[k] = make<T>(0.0);
  T u = make<T>(0.0);
  nonbonded_T<T>(s, x, F, &u, method);
  bonds_T<T>(s, x, F, &u);
  angles_T<T>(s, x, F, &u);
  if (U) *U = u;
}

// Analytic Hessian-vector product H(x) v:
//   pairs and bonds by the 3x3 block A = phi'' rr^T + (phi'/r)(I - rr^T) applied to v_i - v_j;
//   angles by forward-mode dual numbers through the angle force (exact derivative).
void hvp_analytic(const orc_system& s, const double* x, const double* v, double* Hv, int method) {
  const Model m(s);
  const int Q = s.Q;
  for (size_t k = 0; k < 3 * (size_t)Q; ++k) Hv[k] = 0.0;
  auto apply_block = [&](int i, int j, const double* d, double r, double dphi, double d2phi) {
    double u[3] = {v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]};
    double rh[3] = {d[0] / r, d[1] / r, d[2] / r};
    double ru = rh[0] * u[0] + rh[1] * u[1] + rh[2] * u[2];
    for (int k = 0; k < 3; ++k) {
      double au = d2phi * ru * rh[k] + (dphi / r) * (u[k] - ru * rh[k]);
      Hv[3 * i + k] += au;
      Hv[3 * j + k] -= au;
    }
  };
  for_each_pair(s, x, method, [&](int i, int j) {
    const bool ex = m.excluded(i, j);
    if (ex && !m.ewald) return;
    double d[3];
    min_image(s, x + 3 * i, x + 3 * j, d);
    double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double val, dv;
    if (ex) {
      const double qq = kCoulomb * s.charge[i] * s.charge[j];
      m.phi_excl(qq, r, &val, &dv);
      apply_block(i, j, d, r, dv, m.phi_excl2(qq, r));
    } else {
      PairParams p = m.params(i, j);
      m.phi(p, r, &val, &dv);
      apply_block(i, j, d, r, dv, m.phi2(p, r));
    }
  });
  for (int b = 0; b < s.n_bonds; ++b) {
    int i = s.bond_ij[2 * b], j = s.bond_ij[2 * b + 1];
    double d[3];
    min_image(s, x + 3 * i, x + 3 * j, d);
    double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    apply_block(i, j, d, r, s.bond_k[b] * (r - s.bond_r0[b]), s.bond_k[b]);
  }
  if (s.n_angles > 0) {
    // H v = -d/dt F_angles(x + t v) at t = 0, by dual numbers
    std::vector<Dual> xd(3 * (size_t)Q), fd(3 * (size_t)Q, Dual(0.0, 0.0));
    for (size_t k = 0; k < xd.size(); ++k) xd[k] = Dual(x[k], v[k]);
    Dual u(0.0, 0.0);
    angles_T<Dual>(s, xd.data(), fd.data(), &u);
    for (size_t k = 0; k < fd.size(); ++k) Hv[k] -= fd[k].d;
  }
}

}  // namespace

extern "C" {

// U and F at positions x[Q][3]; method 0 = cell list, 1 = brute force. Returns 0.
int orc_forces(const orc_system* s, const double* x, double* F, double* U, int method) {
  forces_T<double>(*s, x, F, U, method);
  return 0;
}

// F(x + i h v) by complex step: real and imaginary parts (either may be NULL), Uc = {Re U, Im U}.
int orc_forces_complex(const orc_system* s, const double* x, const double* v, double h,
                       double* Fre, double* Fim, double* Uc) {
  const size_t n = 3 * (size_t)s->Q;
  std::vector<cplx> xc(n), fc(n);
  for (size_t k = 0; k < n; ++k) xc[k] = cplx(x[k], h * v[k]);
  cplx U;
  forces_T<cplx>(*s, xc.data(), fc.data(), &U, 0);
  for (size_t k = 0; k < n; ++k) {
    if (Fre) Fre[k] = fc[k].real();
    if (Fim) Fim[k] = fc[k].imag();
  }
  if (Uc) { Uc[0] = U.real(); Uc[1] = U.imag(); }
  return 0;
}

// H(x) v.  mode 0 = analytic blocks (+ dual-number angles), 1 = complex step (h = 1e-20),
// 2 = central difference [F(x - h v) - F(x + h v)] / (2h) with the given h.
int orc_hvp(const orc_system* s, const double* x, const double* v, double* Hv, int mode, double h) {
  const size_t n = 3 * (size_t)s->Q;
  if (mode == 0) {
    hvp_analytic(*s, x, v, Hv, 0);
  } else if (mode == 1) {
    const double hc = 1e-20;
    std::vector<double> fim(n);
    orc_forces_complex(s, x, v, hc, nullptr, fim.data(), nullptr);
    for (size_t k = 0; k < n; ++k) Hv[k] = -fim[k] / hc;
  } else {
    std::vector<double> xp(n), xm(n), fp(n), fm(n);
    for (size_t k = 0; k < n; ++k) { xp[k] = x[k] + h * v[k]; xm[k] = x[k] - h * v[k]; }
    forces_T<double>(*s, xp.data(), fp.data(), nullptr, 0);
    forces_T<double>(*s, xm.data(), fm.data(), nullptr, 0);
    for (size_t k = 0; k < n; ++k) Hv[k] = (fm[k] - fp[k]) / (2.0 * h);
  }
  return 0;
}

// Dense Hessian (3Q x 3Q, row major) from analytic HVPs with unit vectors; small Q only.
int orc_hessian_dense(const orc_system* s, const double* x, double* H) {
  const size_t n = 3 * (size_t)s->Q;
  std::vector<double> e(n, 0.0), col(n);
  for (size_t c = 0; c < n; ++c) {
    e[c] = 1.0;
    hvp_analytic(*s, x, e.data(), col.data(), 1);
    for (size_t r = 0; r < n; ++r) H[r * n + c] = col[r];
    e[c] = 0.0;
  }
  return 0;
}

// Effective potential of one path X[N][Q][3] and its gradient.
//   hvp_mode 0: exact gradient with analytic H eta (1: complex-step H eta).
//   hvp_mode 2: the paper's Eq. 5-7 effective forces with the finite-difference term,
//               eps^n = fd_h / max_i |eta^n_i|; G = -F_eff.
// Outputs (any may be NULL): veff[1]; G, F, eta, Heta as [N][Q][3]; parts[2] = {U(R^1), E_spring}.
// For the FD mode Heta holds the FD estimate -[F(R+eps eta) - F(R-eps eta)] / (2 eps).
int orc_veff(const orc_system* s, int N, const double* X, int hvp_mode, double fd_h,
             double* veff, double* G, double* Fout, double* eta_out, double* Heta_out, double* parts) {
  const int Q = s->Q;
  const size_t n3 = 3 * (size_t)Q;
  const double dt = s->dt_path, nu = s->nu_path;
  std::vector<double> K(Q), c(Q);
  for (int i = 0; i < Q; ++i) {
    K[i] = s->mass[i] * nu / (2.0 * dt);       // spring constant (Sec. 1.1)
    c[i] = dt / (s->mass[i] * nu);             // L^n = c F^n (dimensionally consistent reading)
  }
  const int n_force = (N == 1) ? 1 : N - 1;   // bead N needs no force (Eq. 7)
  std::vector<double> F((size_t)N * n3, 0.0), eta((size_t)N * n3, 0.0), Heta((size_t)N * n3, 0.0);
  double U1 = 0.0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int n = 0; n < n_force; ++n) {
    double u;
    forces_T<double>(*s, X + n * n3, F.data() + n * n3, &u, 0);
    if (n == 0) U1 = u;
  }
  // eta^n = R^{n+1} - R^n - L^n
  for (int n = 0; n < N - 1; ++n)
    for (size_t k = 0; k < n3; ++k)
      eta[n * n3 + k] = X[(n + 1) * n3 + k] - X[n * n3 + k] - c[k / 3] * F[n * n3 + k];
  std::vector<double> eps(N, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int n = 0; n < N - 1; ++n) {
    const double* e = eta.data() + n * n3;
    double* he = Heta.data() + n * n3;
    if (hvp_mode == 2) {
      double mx = 0.0;
      for (int i = 0; i < Q; ++i)
        mx = std::max(mx, std::sqrt(e[3 * i] * e[3 * i] + e[3 * i + 1] * e[3 * i + 1] + e[3 * i + 2] * e[3 * i + 2]));
      eps[n] = (mx > 0.0) ? fd_h / mx : fd_h;
      orc_hvp(s, X + n * n3, e, he, 2, eps[n]);
    } else {
      orc_hvp(s, X + n * n3, e, he, hvp_mode == 1 ? 1 : 0, 0.0);
    }
  }
  double Es = 0.0;
  for (int n = 0; n < N - 1; ++n)
    for (int i = 0; i < Q; ++i) {
      const double* e = eta.data() + n * n3 + 3 * i;
      Es += 0.5 * K[i] * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    }
  if (veff) *veff = U1 + Es;
  if (parts) { parts[0] = U1; parts[1] = Es; }
  if (G) {
    for (int n = 0; n < N; ++n)
      for (size_t k = 0; k < n3; ++k) {
        const double Kk = K[k / 3];
        double g;
        if (hvp_mode == 2) {
          // Eqs. 5-7 written out; the FD term [F(R+eps eta)-F(R-eps eta)]/(4 eps) = -Heta/2
          const double fd = -0.5 * Heta[n * n3 + k];
          double feff;
          if (N == 1) {
            feff = F[k];
          } else if (n == 0) {                                     // Eq. 6
            feff = 0.5 * F[k] + Kk * (X[n3 + k] - X[k]) + fd;
          } else if (n == N - 1) {                                 // Eq. 7
            feff = -Kk * (X[n * n3 + k] - X[(n - 1) * n3 + k]) + 0.5 * F[(n - 1) * n3 + k];
          } else {                                                 // Eq. 5
            feff = -Kk * (2.0 * X[n * n3 + k] - X[(n - 1) * n3 + k] - X[(n + 1) * n3 + k]) +
                   0.5 * (F[(n - 1) * n3 + k] - F[n * n3 + k]) + fd;
          }
          g = -feff;
        } else {
          g = 0.0;
          if (n == 0) g -= F[k];
          if (n > 0) g += Kk * eta[(n - 1) * n3 + k];
          if (n < N - 1) g += -Kk * eta[n * n3 + k] + 0.5 * Heta[n * n3 + k];
        }
        G[n * n3 + k] = g;
      }
  }
  if (Fout) std::memcpy(Fout, F.data(), sizeof(double) * N * n3);
  if (eta_out) std::memcpy(eta_out, eta.data(), sizeof(double) * N * n3);
  if (Heta_out) std::memcpy(Heta_out, Heta.data(), sizeof(double) * N * n3);
  return 0;
}

// Im V_eff(X + i h D) / h: the exact directional derivative of V_eff along D (complex step).
int orc_veff_complex_dir(const orc_system* s, int N, const double* X, const double* D, double h, double* out) {
  const int Q = s->Q;
  const size_t n3 = 3 * (size_t)Q;
  const double dt = s->dt_path, nu = s->nu_path;
  std::vector<cplx> Xc((size_t)N * n3), F((size_t)N * n3);
  for (size_t k = 0; k < Xc.size(); ++k) Xc[k] = cplx(X[k], h * D[k]);
  const int n_force = (N == 1) ? 1 : N - 1;
  std::vector<cplx> U(n_force);
#pragma omp parallel for schedule(dynamic, 1)
  for (int n = 0; n < n_force; ++n) forces_T<cplx>(*s, Xc.data() + n * n3, F.data() + n * n3, &U[n], 0);
  cplx V = U[0];
  for (int n = 0; n < N - 1; ++n)
    for (size_t k = 0; k < n3; ++k) {
      const double m = s->mass[k / 3];
      cplx e = Xc[(n + 1) * n3 + k] - Xc[n * n3 + k] - (dt / (m * nu)) * F[n * n3 + k];
      V += 0.5 * (m * nu / (2.0 * dt)) * e * e;
    }
  *out = V.imag() / h;
  return 0;
}

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32 Philox S-box
// with the Weyl key schedule.
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

// Three standard normals for (seed, step, bead, atom) by Box-Muller on one Philox block:
// counter = {atom, bead, step_lo, step_hi}, key = {seed_lo, seed_hi};
// u1 = (w0 + 1) 2^-32 in (0, 1], u2 = w1 2^-32, likewise (w2, w3).
void orc_gauss3(uint64_t seed, uint64_t step, uint32_t bead, uint32_t atom, double out[3]) {
  uint32_t ctr[4] = {atom, bead, (uint32_t)step, (uint32_t)(step >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  const double two32 = 4294967296.0;
  const double pi = 3.14159265358979323846;
  double u1 = ((double)w[0] + 1.0) / two32, u2 = (double)w[1] / two32;
  double u3 = ((double)w[2] + 1.0) / two32, u4 = (double)w[3] / two32;
  double r1 = std::sqrt(-2.0 * std::log(u1)), r2 = std::sqrt(-2.0 * std::log(u3));
  out[0] = r1 * std::cos(2.0 * pi * u2);
  out[1] = r1 * std::sin(2.0 * pi * u2);
  out[2] = r2 * std::cos(2.0 * pi * u4);
}

// Collective variable of the bias: s = |c_A - c_B| (minimum image), with each centroid taken
// over its group unwrapped relative to the group's first atom.  w * ds/dx is added into
// dsdx[Q][3] (if non-NULL); returns s.
double orc_cv_distance(const orc_system* s, const double* x, const int32_t* ga, int na,
                       const int32_t* gb, int nb, double* dsdx, double w) {
  double ca[3] = {0, 0, 0}, cb[3] = {0, 0, 0};
  for (int k = 0; k < na; ++k) {
    double d[3];
    min_image(*s, x + 3 * ga[k], x + 3 * ga[0], d);
    for (int c = 0; c < 3; ++c) ca[c] += (x[3 * ga[0] + c] + d[c]) / na;
  }
  for (int k = 0; k < nb; ++k) {
    double d[3];
    min_image(*s, x + 3 * gb[k], x + 3 * gb[0], d);
    for (int c = 0; c < 3; ++c) cb[c] += (x[3 * gb[0] + c] + d[c]) / nb;
  }
  double d[3];
  min_image(*s, ca, cb, d);
  double sv = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (dsdx) {
    for (int k = 0; k < na; ++k)
      for (int c = 0; c < 3; ++c) dsdx[3 * ga[k] + c] += w * d[c] / sv / na;
    for (int k = 0; k < nb; ++k)
      for (int c = 0; c < 3; ++c) dsdx[3 * gb[k] + c] -= w * d[c] / sv / nb;
  }
  return sv;
}

// Metadynamics bias (Sec. 1.2) on S = s(R^N) (e2e = 0) or S = s(R^N) - s(R^1) (e2e = 1, Eq. 8):
// V_b = sum_k h_k exp(-(S - S_k)^2 / (2 w_k^2)).  Adds dV_b/dX to G[N][Q][3] (if non-NULL).
// Returns V_b; *cv receives S.
double orc_bias(const orc_system* s, int N, const double* X, const int32_t* ga, int na,
                const int32_t* gb, int nb, int e2e, int n_gauss, const double* centers,
                const double* heights, const double* widths, double* G, double* cv) {
  const size_t n3 = 3 * (size_t)s->Q;
  std::vector<double> dS((size_t)N * n3, 0.0);
  double S = orc_cv_distance(s, X + (size_t)(N - 1) * n3, ga, na, gb, nb, dS.data() + (size_t)(N - 1) * n3, 1.0);
  if (e2e) S -= orc_cv_distance(s, X, ga, na, gb, nb, dS.data(), -1.0);
  double V = 0.0, dV = 0.0;
  for (int k = 0; k < n_gauss; ++k) {
    const double z = (S - centers[k]) / widths[k];
    const double e = heights[k] * std::exp(-0.5 * z * z);
    V += e;
    dV += -e * z / widths[k];
  }
  if (G)
    for (size_t k = 0; k < dS.size(); ++k) G[k] += dV * dS[k];
  if (cv) *cv = S;
  return V;
}

// Collective variable with optional mass weighting: s = |C_A - C_B| (minimum image), where
// C = sum_k w_k x_k / sum_k w_k over a group, w_k = m_k when com != 0 (the centre-of-mass
// distance the paper biases, Sec. 3) and 1 otherwise (the geometric centroid); each atom is
// unwrapped relative to its group's first atom.  Adds w * ds/dx into dsdx[Q][3] (if non-NULL);
// returns s.
double orc_cv_com(const orc_system* s, const double* x, const int32_t* ga, int na, const int32_t* gb,
                  int nb, int com, double* dsdx, double w) {
  auto centre = [&](const int32_t* g, int n, double* c, double* W) {
    double acc[3] = {0, 0, 0}, wt = 0.0;
    for (int k = 0; k < n; ++k) {
      double d[3];
      min_image(*s, x + 3 * g[k], x + 3 * g[0], d);
      const double m = com ? s->mass[g[k]] : 1.0;
      for (int c2 = 0; c2 < 3; ++c2) acc[c2] += m * (x[3 * g[0] + c2] + d[c2]);
      wt += m;
    }
    for (int c2 = 0; c2 < 3; ++c2) c[c2] = acc[c2] / wt;
    *W = wt;
  };
  double ca[3], cb[3], Wa, Wb;
  centre(ga, na, ca, &Wa);
  centre(gb, nb, cb, &Wb);
  double d[3];
  min_image(*s, ca, cb, d);
  const double sv = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (dsdx) {
    for (int k = 0; k < na; ++k) {
      const double m = com ? s->mass[ga[k]] : 1.0;
      for (int c = 0; c < 3; ++c) dsdx[3 * ga[k] + c] += w * d[c] / sv * m / Wa;
    }
    for (int k = 0; k < nb; ++k) {
      const double m = com ? s->mass[gb[k]] : 1.0;
      for (int c = 0; c < 3; ++c) dsdx[3 * gb[k] + c] -= w * d[c] / sv * m / Wb;
    }
  }
  return sv;
}

// Bias of orc_bias on the CV of orc_cv_com (com selects the mass weighting).
double orc_bias_com(const orc_system* s, int N, const double* X, const int32_t* ga, int na,
                    const int32_t* gb, int nb, int e2e, int com, int n_gauss, const double* centers,
                    const double* heights, const double* widths, double* G, double* cv) {
  const size_t n3 = 3 * (size_t)s->Q;
  std::vector<double> dS((size_t)N * n3, 0.0);
  double S = orc_cv_com(s, X + (size_t)(N - 1) * n3, ga, na, gb, nb, com, dS.data() + (size_t)(N - 1) * n3, 1.0);
  if (e2e) S -= orc_cv_com(s, X, ga, na, gb, nb, com, dS.data(), -1.0);
  double V = 0.0, dV = 0.0;
  for (int k = 0; k < n_gauss; ++k) {
    const double z = (S - centers[k]) / widths[k];
    const double e = heights[k] * std::exp(-0.5 * z * z);
    V += e;
    dV += -e * z / widths[k];
  }
  if (G)
    for (size_t k = 0; k < dS.size(); ++k) G[k] += dV * dS[k];
  if (cv) *cv = S;
  return V;
}

// Multi-CV bias: n_cv CVs S_d (each the CV of orc_bias_com on its own groups, with its own
// e2e and com flags; the groups of CV d are ga[ga_off[d] .. ga_off[d + 1]) and likewise gb) and
// V_b = sum_k h_k exp(-sum_d (S_d - c_kd)^2 / (2 w_kd^2)), centres and widths [n_gauss][n_cv].
// Adds dV_b/dX to G (if non-NULL); cv[n_cv] (if non-NULL) receives the S_d.  Returns V_b.
double orc_bias_multi(const orc_system* s, int N, const double* X, int n_cv, const int32_t* ga,
                      const int32_t* ga_off, const int32_t* gb, const int32_t* gb_off, const int32_t* e2e,
                      const int32_t* com, int n_gauss, const double* centers, const double* widths,
                      const double* heights, double* G, double* cv) {
  const size_t n3 = 3 * (size_t)s->Q;
  std::vector<std::vector<double>> dS(n_cv, std::vector<double>((size_t)N * n3, 0.0));
  std::vector<double> S(n_cv), dV(n_cv, 0.0);
  for (int d = 0; d < n_cv; ++d) {
    const int32_t* a = ga + ga_off[d];
    const int32_t* b = gb + gb_off[d];
    const int na = ga_off[d + 1] - ga_off[d], nb = gb_off[d + 1] - gb_off[d];
    S[d] = orc_cv_com(s, X + (size_t)(N - 1) * n3, a, na, b, nb, com[d], dS[d].data() + (size_t)(N - 1) * n3, 1.0);
    if (e2e[d]) S[d] -= orc_cv_com(s, X, a, na, b, nb, com[d], dS[d].data(), -1.0);
  }
  double V = 0.0;
  for (int k = 0; k < n_gauss; ++k) {
    double q = 0.0;
    for (int d = 0; d < n_cv; ++d) {
      const double z = (S[d] - centers[(size_t)k * n_cv + d]) / widths[(size_t)k * n_cv + d];
      q += z * z;
    }
    const double e = heights[k] * std::exp(-0.5 * q);
    V += e;
    for (int d = 0; d < n_cv; ++d) {
      const double w = widths[(size_t)k * n_cv + d];
      dV[d] += -e * (S[d] - centers[(size_t)k * n_cv + d]) / (w * w);
    }
  }
  if (G)
    for (int d = 0; d < n_cv; ++d)
      for (size_t k = 0; k < dS[d].size(); ++k) G[k] += dV[d] * dS[d][k];
  if (cv)
    for (int d = 0; d < n_cv; ++d) cv[d] = S[d];
  return V;
}

}  // extern "C"

namespace {

// One BAOAB step (gamma > 0) or velocity-Verlet step (gamma = 0) of the path dynamics
// M d2R^n/dt2 = -dU_tot/dR^n (Eq. 4) with fictitious masses equal to the physical ones: half
// kick, half drift, Ornstein-Uhlenbeck velocity update with Philox noise keyed by (seed, step,
// bead, atom), half drift, new gradient, half kick.  grad(Xe, G) returns U_tot at Xe and writes
// its gradient; Xe is X rounded to float32 when round_f32 != 0.
double baoab_step(const orc_system* s, int N, double* X, double* Vel, double* G, double dt, double gamma,
                  double temperature, uint64_t seed, uint64_t step, int round_f32,
                  const std::function<double(const double*, double*)>& grad) {
  const int Q = s->Q;
  const size_t n3 = 3 * (size_t)Q, tot = (size_t)N * n3;
  const double kT = kBoltzmann * temperature;
  for (size_t k = 0; k < tot; ++k) Vel[k] -= 0.5 * dt * G[k] / s->mass[(k % n3) / 3];
  for (size_t k = 0; k < tot; ++k) X[k] += 0.5 * dt * Vel[k];
  if (gamma > 0.0) {
    const double c1 = std::exp(-gamma * dt);
    const double c2 = std::sqrt(1.0 - c1 * c1);
    for (int n = 0; n < N; ++n)
      for (int i = 0; i < Q; ++i) {
        double g[3];
        orc_gauss3(seed, step, (uint32_t)n, (uint32_t)i, g);
        const double sd = c2 * std::sqrt(kT / s->mass[i]);
        for (int c = 0; c < 3; ++c) {
          double& v = Vel[n * n3 + 3 * i + c];
          v = c1 * v + sd * g[c];
        }
      }
  }
  for (size_t k = 0; k < tot; ++k) X[k] += 0.5 * dt * Vel[k];
  std::vector<double> Xe(X, X + tot);
  if (round_f32)
    for (auto& v : Xe) v = (double)(float)v;
  const double V = grad(Xe.data(), G);
  for (size_t k = 0; k < tot; ++k) Vel[k] -= 0.5 * dt * G[k] / s->mass[(k % n3) / 3];
  return V;
}

}  // namespace

extern "C" {

// One step of the path dynamics on V_eff alone (see baoab_step).  X, Vel: [N][Q][3] FP64 state,
// updated in place; G: gradient at X on entry, at the new X on exit.  Returns V_eff at the new
// positions.
double orc_step(const orc_system* s, int N, double* X, double* Vel, double* G, double dt, double gamma,
                double temperature, uint64_t seed, uint64_t step, int round_f32) {
  return baoab_step(s, N, X, Vel, G, dt, gamma, temperature, seed, step, round_f32,
                    [&](const double* Xe, double* Gout) {
                      double V;
                      orc_veff(s, N, Xe, 0, 0.0, &V, Gout, nullptr, nullptr, nullptr, nullptr);
                      return V;
                    });
}

// Metadynamics of paths (Sec. 1.2 with the deposition of Sec. 3, a new Gaussian every `stride`
// MD steps): n_deposits rounds of `stride` steps of the path dynamics on V_eff + V_bias, each
// round ending with one Gaussian of the given height and width centred at the CV's value at the
// current (float32-rounded when round_f32) positions.  After each deposit the gradient is
// evaluated again, so the next step starts from the new bias.  Step k of the run draws its
// noise with counter step0 + k.  centers/heights/widths hold n_gauss0 Gaussians on entry and
// n_gauss0 + n_deposits on exit.  Vel holds the velocities (zero for a fresh start).  Returns
// V_eff + V_bias at the final positions.
double orc_metad(const orc_system* s, int N, double* X, double* Vel, double dt, double gamma, double temperature,
                 uint64_t seed, uint64_t step0, int n_deposits, int stride, const int32_t* ga, int na,
                 const int32_t* gb, int nb, int e2e, int com, double height, double width, int n_gauss0,
                 double* centers, double* heights, double* widths, int round_f32) {
  const size_t tot = (size_t)N * 3 * (size_t)s->Q;
  int ng = n_gauss0;
  auto total = [&](const double* Xe, double* Gout) {
    double V;
    orc_veff(s, N, Xe, 0, 0.0, &V, Gout, nullptr, nullptr, nullptr, nullptr);
    return V + orc_bias_com(s, N, Xe, ga, na, gb, nb, e2e, com, ng, centers, heights, widths, Gout, nullptr);
  };
  auto rounded = [&](const double* x) {
    std::vector<double> Xe(x, x + tot);
    if (round_f32)
      for (auto& v : Xe) v = (double)(float)v;
    return Xe;
  };
  std::vector<double> G(tot);
  double V = total(rounded(X).data(), G.data());
  uint64_t step = step0;
  for (int d = 0; d < n_deposits; ++d) {
    for (int k = 0; k < stride; ++k)
      V = baoab_step(s, N, X, Vel, G.data(), dt, gamma, temperature, seed, step++, round_f32, total);
    const std::vector<double> Xe = rounded(X);
    double S = 0.0;
    orc_bias_com(s, N, Xe.data(), ga, na, gb, nb, e2e, com, 0, nullptr, nullptr, nullptr, nullptr, &S);
    centers[ng] = S;
    heights[ng] = height;
    widths[ng] = width;
    ++ng;
    V = total(Xe.data(), G.data());
  }
  return V;
}

// Metadynamics of paths on n_cv CVs (orc_metad with the bias of orc_bias_multi): each deposit
// is centred at the current S_d, with height `height` and widths dep_widths[d].  centers and
// widths are [n_gauss0 + n_deposits][n_cv], heights [n_gauss0 + n_deposits].
double orc_metad_multi(const orc_system* s, int N, double* X, double* Vel, double dt, double gamma,
                       double temperature, uint64_t seed, uint64_t step0, int n_deposits, int stride, int n_cv,
                       const int32_t* ga, const int32_t* ga_off, const int32_t* gb, const int32_t* gb_off,
                       const int32_t* e2e, const int32_t* com, double height, const double* dep_widths,
                       int n_gauss0, double* centers, double* widths, double* heights, int round_f32) {
  const size_t tot = (size_t)N * 3 * (size_t)s->Q;
  int ng = n_gauss0;
  auto total = [&](const double* Xe, double* Gout) {
    double V;
    orc_veff(s, N, Xe, 0, 0.0, &V, Gout, nullptr, nullptr, nullptr, nullptr);
    return V + orc_bias_multi(s, N, Xe, n_cv, ga, ga_off, gb, gb_off, e2e, com, ng, centers, widths, heights,
                              Gout, nullptr);
  };
  auto rounded = [&](const double* x) {
    std::vector<double> Xe(x, x + tot);
    if (round_f32)
      for (auto& v : Xe) v = (double)(float)v;
    return Xe;
  };
  std::vector<double> G(tot), Snow(n_cv);
  double V = total(rounded(X).data(), G.data());
  uint64_t step = step0;
  for (int dep = 0; dep < n_deposits; ++dep) {
    for (int k = 0; k < stride; ++k)
      V = baoab_step(s, N, X, Vel, G.data(), dt, gamma, temperature, seed, step++, round_f32, total);
    const std::vector<double> Xe = rounded(X);
    orc_bias_multi(s, N, Xe.data(), n_cv, ga, ga_off, gb, gb_off, e2e, com, 0, nullptr, nullptr, nullptr, nullptr,
                   Snow.data());
    for (int d = 0; d < n_cv; ++d) {
      centers[(size_t)ng * n_cv + d] = Snow[d];
      widths[(size_t)ng * n_cv + d] = dep_widths[d];
    }
    heights[ng] = height;
    ++ng;
    V = total(Xe.data(), G.data());
  }
  return V;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
