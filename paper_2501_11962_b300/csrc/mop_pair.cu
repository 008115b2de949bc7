// Cluster-pair kernels of the hot path: nonbonded force F(R^n), adjoint Hessian-vector product
// H(R^n) eta^n, and the paper's finite-difference stand-in F(R + eps eta) - F(R - eps eta).
// These run the FP64 mode (MOP_PREC_FP64, config 1) and, selected with MOP_PAIR_KERNELS=half, the
// half-list form of the mixed mode; mixed precision otherwise runs the bead-lane kernels of
// mop_pairb.cu.
//
// Paper: the three do_force calls per bead of Sec. 2.1 (Fig. 2) carry "the majority of the
// computational effort"; the FD term is the last term of Eq. 5.  One launch covers every (path,
// bead, i-cluster) unit of every path.
//
// Work unit = one warp x one i-cluster (8 atoms) x B beads (FP64: 1; FP32: 2, in f32x2).  Lane l
// handles i-atom (l & 7) against j-atoms (l >> 3) and (l >> 3) + 4 of each listed j-cluster.
// FP64 mode walks the full list (every cluster pair from both sides), so each i-atom's sum is
// complete in its own warp and nothing else is written.  The FP32 half-list form walks each
// unordered cluster pair once: the j-atoms' share (-f) is summed over the warp and added to
// jacc as 2^-23 fixed point with 64-bit integer atomics (order-independent, so the result is
// bitwise reproducible).  FP32 partial sums over 16 j-clusters are folded into an FP32 (hi, lo)
// pair by TwoSum, and the four lanes of an i-atom are summed as double-floats (FP64 mode sums in
// FP64).  Pair potential (r < rc, shifted-force modifier by default):
//   phi(r) = c12 r^-12 - c6 r^-6 + f q_i q_j (1/r + k_rf r^2 - c_rf)
//   g  = -phi'_sf(r)/r                     force on i: g d,  d = r_i - r_j
//   b  = (phi''(r) + g) / r^2              H block A = b d d^T - g I,  A u with u = eta_i - eta_j
#include "mop_host.h"
#include "mop_pairmath.cuh"

// resident 128-thread blocks per SM requested for the FP32 pair kernels (register budget)
#ifndef MOP_PAIR_MINB
#define MOP_PAIR_MINB 4
#endif


namespace mop {
namespace {

template <class R> struct Tr;

template <> struct Tr<float> {
  using V4 = float4;
  using E4 = float4;   // eta as stored for the pair kernels
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ const V4* xq(const PathDev& P) { return P.xq; }
  static __device__ __forceinline__ void delta(const PathDev&, size_t, const int4& en, float* D) {
    D[0] = __int_as_float(en.y);
    D[1] = __int_as_float(en.z);
    D[2] = __int_as_float(en.w);
  }
  static __device__ __forceinline__ void eta(const PathDev& P, size_t k, float* u) {
    const float4 v = __ldg(&P.eta32[k]);
    u[0] = v.x;
    u[1] = v.y;
    u[2] = v.z;
  }
  static __device__ __forceinline__ V4 tab(const SysConsts& sc, int k) { return sc.tab[k]; }
};

template <> struct Tr<double> {
  using V4 = double4_32a;
  static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
  static __device__ __forceinline__ const V4* xq(const PathDev& P) { return P.xq64; }
  static __device__ __forceinline__ void delta(const PathDev& P, size_t e, const int4&, double* D) {
    const double4_32a v = P.ent64[e];
    D[0] = v.x;
    D[1] = v.y;
    D[2] = v.z;
  }
  static __device__ __forceinline__ void eta(const PathDev& P, size_t k, double* u) {
    u[0] = P.eta[3 * k];
    u[1] = P.eta[3 * k + 1];
    u[2] = P.eta[3 * k + 2];
  }
  static __device__ __forceinline__ V4 tab(const SysConsts& sc, int k) { return sc.tab64[k]; }
};

// Three-component accumulator: FP32 chunk sums folded into (hi, lo) by TwoSum, or plain FP64.
template <class R> struct Acc3;
template <> struct Acc3<float> {
  float a[3] = {0.f, 0.f, 0.f}, h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      two_sum_add(h[k], l[k], a[k]);
      a[k] = 0.f;
    }
  }
  __device__ __forceinline__ double get(int k) const { return ((double)h[k] + (double)l[k]) + (double)a[k]; }
};
template <> struct Acc3<double> {
  double a[3] = {0.0, 0.0, 0.0};
  __device__ __forceinline__ void fold() {}
  __device__ __forceinline__ double get(int k) const { return a[k]; }
};
template <class R> struct Acc1;
template <> struct Acc1<float> {
  float a = 0.f, h = 0.f, l = 0.f;
  __device__ __forceinline__ void fold() { two_sum_add(h, l, a); a = 0.f; }
  __device__ __forceinline__ double get() const { return ((double)h + (double)l) + (double)a; }
};
template <> struct Acc1<double> {
  double a = 0.0;
  __device__ __forceinline__ void fold() {}
  __device__ __forceinline__ double get() const { return a; }
};

template <class R> struct Cst {
  R rc, rc2, krf, crf, k2rf, drf;
  R ewb, ewb2, ewc2, ewec;   // Ewald: beta, beta^2, 2 beta / sqrt(pi), erfc(beta rc) / rc
  __device__ __forceinline__ explicit Cst(const SysConsts& sc);
};
template <> __device__ __forceinline__ Cst<float>::Cst(const SysConsts& sc)
    : rc(sc.rcf), rc2(sc.rc2f), krf(sc.krff), crf(sc.crff), k2rf(sc.k2rff), drf(sc.drff), ewb(sc.ewb),
      ewb2(sc.ewb2), ewc2(sc.ewc2), ewec(sc.ewec) {}
template <> __device__ __forceinline__ Cst<double>::Cst(const SysConsts& sc)
    : rc(sc.rc), rc2(sc.rc2), krf(sc.krf), crf(sc.crf), k2rf(sc.k2rf), drf(sc.drf), ewb(0), ewb2(0), ewc2(0),
      ewec(0) {}

// g = -phi'_sf(r)/r from r^-1 powers; p = (12 c12, 6 c6, phi'_LJ(rc), phi_LJ(rc)), sh = phi'(rc)
template <class R, class V4>
__device__ __forceinline__ R pair_g(R rinv, R rinv2, R rinv6, const V4& p, R qq, R sh, R k2rf) {
  return rinv6 * fma(p.x, rinv6, -p.y) * rinv2 + qq * fma(rinv, rinv2, -k2rf) + sh * rinv;
}

// Per (entry, half) constants shared by all beads of a unit: type-pair row p = (12 c12, 6 c6,
// phi'_LJ(rc), phi_LJ(rc)), qq = f q_i q_j, sh = phi'(rc), and derived factors.
template <class R> struct PairK {
  R A, B;      // 12 c12, 6 c6
  R qq, sh;    // f q_i q_j, phi'(rc) of the pair
  R qk;        // qq * 2 k_rf
  R A14, B8;   // 14 * 12 c12, 8 * 6 c6   (HVP)
  R q3;        // 3 qq                    (HVP)
  R Ew;        // phi_LJ(rc)              (energy)
};

template <class R, int MODE, class V4>
__device__ __forceinline__ PairK<R> pair_consts(const Cst<R>& k, const V4& p, R qq) {
  PairK<R> c;
  c.A = p.x;
  c.B = p.y;
  c.qq = qq;
  c.sh = fma(qq, k.drf, p.z);
  c.qk = qq * k.k2rf;
  if (MODE == 1) {
    c.A14 = R(14) * p.x;
    c.B8 = R(8) * p.y;
    c.q3 = R(3) * qq;
  }
  c.Ew = p.w;
  return c;
}

// g = -phi'_sf(r) / r = r^-2 [r^-6 (A r^-6 - B) + qq r^-1] + (sh r^-1 - qq 2 k_rf)
template <class R>
__device__ __forceinline__ R pair_g2(const PairK<R>& c, R rinv, R rinv2, R rinv6) {
  const R t = fma(c.qq, rinv, rinv6 * fma(c.A, rinv6, -c.B));
  return fma(rinv2, t, fma(c.sh, rinv, -c.qk));
}

// One pair for one bead (i-atom of this lane at xs, j-atom xj); cutoff test against rc2e
// (negative for an excluded pair).  Accumulates F (MODE 0), H eta (MODE 1) or F(+) - F(-)
// (MODE 2) into a[3] and the pair energy into e (ENERGY).
// Ewald real space (EW): the electrostatic factor of g, qq (erfc(beta r)/r + 2 beta/sqrt(pi)
// exp(-beta^2 r^2)), from erfc(x) = exp(-x^2) erfcx(x) (erfcx_rational of mop_pairmath.cuh).
template <class R>
__device__ __forceinline__ void ewald_terms(const Cst<R>& k, R r2, R rinv, R* ec, R* c2e) {
  const R G = __expf(-k.ewb2 * r2);
  *ec = G * erfcx_rational(k.ewb * (r2 * rinv));
  *c2e = k.ewc2 * G;
}

// g = -phi'_sf(r) / r with Ewald real space: r^-2 [r^-6 (A r^-6 - B) + qq (ec r^-1 + c2E)] + sh r^-1
template <class R>
__device__ __forceinline__ R pair_g2_ew(const PairK<R>& c, R rinv, R rinv2, R rinv6, R ec, R c2e) {
  const R t = fma(c.qq, fma(ec, rinv, c2e), rinv6 * fma(c.A, rinv6, -c.B));
  return fma(rinv2, t, c.sh * rinv);
}

// HALF: the pair's contribution to atom i is also returned in f (atom j receives -f).
// EW: Ewald real-space electrostatics instead of the reaction field.
template <class R, int MODE, bool ENERGY, bool HALF, bool EW, class V4>
__device__ __forceinline__ void pair_one(const Cst<R>& k, const PairK<R>& c, R xs, R ys, R zs, const V4& xj, R rc2e,
                                         const R* ei, const R* ej, R eps, R ew, R* a, R& e, R* f) {
  const R dx = xs - xj.x, dy = ys - xj.y, dz = zs - xj.z;
  if (MODE == 0) {
    const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const bool in = r2 < rc2e;
    const R rinv = Tr<R>::rsq(r2);
    const R rinv2 = rinv * rinv;
    const R rinv6 = rinv2 * rinv2 * rinv2;
    R ec = R(0), c2e = R(0);
    if (EW) ewald_terms<R>(k, r2, rinv, &ec, &c2e);
    R g = EW ? pair_g2_ew<R>(c, rinv, rinv2, rinv6, ec, c2e) : pair_g2<R>(c, rinv, rinv2, rinv6);
    g = in ? g : R(0);
    if (HALF) {
      f[0] = g * dx;
      f[1] = g * dy;
      f[2] = g * dz;
      a[0] += f[0];
      a[1] += f[1];
      a[2] += f[2];
    } else {
      a[0] = fma(g, dx, a[0]);
      a[1] = fma(g, dy, a[1]);
      a[2] = fma(g, dz, a[2]);
    }
    if (ENERGY) {
      // phi(r) - phi(rc) - (r - rc) phi'(rc); phi_RF(rc) = 0 by the choice of c_rf
      const R r = r2 * rinv;
      const R elj = rinv6 * fma(c.A * R(1.0 / 12.0), rinv6, -c.B * R(1.0 / 6.0));
      const R erf = EW ? c.qq * fma(ec, rinv, -k.ewec) : c.qq * (rinv + fma(k.krf, r2, -k.crf));
      const R E = elj + erf - c.Ew - (r - k.rc) * c.sh;
      e = in ? fma(ew, E, e) : e;
    }
  } else if (MODE == 1) {
    const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const bool in = r2 < rc2e;
    const R ux = ei[0] - ej[0], uy = ei[1] - ej[1], uz = ei[2] - ej[2];
    const R rinv = Tr<R>::rsq(r2);
    const R rinv2 = rinv * rinv;
    const R rinv3 = rinv * rinv2;
    const R rinv6 = rinv2 * rinv2 * rinv2;
    R g, b;
    if (EW) {
      // b = r^-4 r^-6 (14 A r^-6 - 8 B) + r^-3 [qq (3 ec r^-2 + c2E (3 r^-1 + 2 beta^2 r)) + sh]
      R ec, c2e;
      ewald_terms<R>(k, r2, rinv, &ec, &c2e);
      g = pair_g2_ew<R>(c, rinv, rinv2, rinv6, ec, c2e);
      const R el = fma(R(3) * ec, rinv2, c2e * fma(R(2) * k.ewb2, r2 * rinv, R(3) * rinv));
      b = fma(rinv2 * rinv2, rinv6 * fma(c.A14, rinv6, -c.B8), rinv3 * fma(c.qq, el, c.sh));
    } else {
      g = pair_g2<R>(c, rinv, rinv2, rinv6);
      // b = (phi'' + g) / r^2 = r^-4 r^-6 (14 A r^-6 - 8 B) + r^-3 (3 qq r^-2 + sh)
      b = fma(rinv2 * rinv2, rinv6 * fma(c.A14, rinv6, -c.B8), rinv3 * fma(c.q3, rinv2, c.sh));
    }
    const R s = fma(dx, ux, fma(dy, uy, dz * uz));
    const R t = in ? b * s : R(0);
    const R ng = in ? -g : R(0);
    if (HALF) {
      f[0] = fma(ng, ux, t * dx);
      f[1] = fma(ng, uy, t * dy);
      f[2] = fma(ng, uz, t * dz);
      a[0] += f[0];
      a[1] += f[1];
      a[2] += f[2];
    } else {
      a[0] = fma(ng, ux, fma(t, dx, a[0]));
      a[1] = fma(ng, uy, fma(t, dy, a[1]));
      a[2] = fma(ng, uz, fma(t, dz, a[2]));
    }
  } else {
    const R ux = eps * (ei[0] - ej[0]), uy = eps * (ei[1] - ej[1]), uz = eps * (ei[2] - ej[2]);
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      const R px = sgn ? dx - ux : dx + ux, py = sgn ? dy - uy : dy + uy, pz = sgn ? dz - uz : dz + uz;
      const R r2 = fma(px, px, fma(py, py, pz * pz));
      const bool in = r2 < rc2e;
      const R rinv = Tr<R>::rsq(r2);
      const R rinv2 = rinv * rinv;
      const R rinv6 = rinv2 * rinv2 * rinv2;
      R g;
      if (EW) {
        R ec, c2e;
        ewald_terms<R>(k, r2, rinv, &ec, &c2e);
        g = pair_g2_ew<R>(c, rinv, rinv2, rinv6, ec, c2e);
      } else {
        g = pair_g2<R>(c, rinv, rinv2, rinv6);
      }
      g = in ? (sgn ? -g : g) : R(0);
      if (HALF) {
        f[0] = sgn ? fma(g, px, f[0]) : g * px;
        f[1] = sgn ? fma(g, py, f[1]) : g * py;
        f[2] = sgn ? fma(g, pz, f[2]) : g * pz;
      } else {
        a[0] = fma(g, px, a[0]);
        a[1] = fma(g, py, a[1]);
        a[2] = fma(g, pz, a[2]);
      }
    }
    if (HALF) {
      a[0] += f[0];
      a[1] += f[1];
      a[2] += f[2];
    }
  }
}

// ---- two beads per instruction (FP32 mode) ------------------------------------------------
// A lane evaluates the same (i, j) pair for the two beads of its unit with the same pair
// constants, so the FP32 arithmetic of both runs in packed f32x2 instructions (fma/add/mul.f32x2,
// sm_100 family): half the issue slots for the same FMA-pipe work.  Only rsqrt, exp2, the
// reciprocal and the cutoff selects stay per bead.  x = bead n0, y = bead n0 + 1.
#ifndef MOP_PACK2
#define MOP_PACK2 1
#endif
// packed units may stage each j-atom with its two beads interleaved, (x, x', y, y') and
// (z, z', q, q), so that 128-bit shared-memory reads deliver ready f32x2 operands
#ifndef MOP_ILV
#define MOP_ILV 1
#endif
// packed units skip a listed half with no pair within rc in either bead (warp vote); FD units
// with the radius rc + 2 h of their displaced pairs
#ifndef MOP_SKIP
#define MOP_SKIP 1
#endif
// adjoint H eta kernels read the j eta after the skip vote (H eta -0.09 ms, Ewald H eta
// -0.32 ms on the 150k-atom path; the FD kernels measured 1% slower that way and read it before)
#ifndef MOP_EJ_LATE
#define MOP_EJ_LATE 1
#endif
#ifndef MOP_SPTR
#define MOP_SPTR 1   // HVP and FD kernels: the j fetch's base pointers in shared memory
#endif
// pair constants of one (entry, half) duplicated into both lanes of the f32x2 operands
struct PairK2 {
  float2 A, nB, qq, sh, nqk;   // 12 c12, -6 c6, f qi qj, phi'(rc), -qq 2 k_rf
  float2 A14, nB8, q3;         // HVP: 14 * 12 c12, -8 * 6 c6, 3 qq
};

template <int MODE>
__device__ __forceinline__ PairK2 pair_consts2(const PairK<float>& c) {
  PairK2 d;
  d.A = dup2(c.A);
  d.nB = dup2(-c.B);
  d.qq = dup2(c.qq);
  d.sh = dup2(c.sh);
  d.nqk = dup2(-c.qk);
  if (MODE == 1) {
    d.A14 = dup2(c.A14);
    d.nB8 = dup2(-c.B8);
    d.q3 = dup2(c.q3);
  }
  return d;
}

// Ewald: erfc(beta r) and the force term 2 beta/sqrt(pi) G for both beads
__device__ __forceinline__ void ewald_terms2(const Cst<float>& k, float2 r2, float2 rinv, float2* ec, float2* c2e) {
  ewald_terms2(k.ewb, k.ewb2, k.ewc2, r2, rinv, ec, c2e);
}

// One pair for both beads of the unit (HALF list): MODE 0 force, MODE 1 adjoint H eta.  xs and
// xj: the i- and j-atom per dimension (bead x, bead y), one of them shifted by the entry's Delta;
// ei/ej eta (MODE 1).  Adds the i-side term to a and returns it in f.  ENERGY: also adds ew times
// the pair energy of bead x (the first bead of the unit) to e.
// pair_two_d takes the separation d = xs - xj and r2 = |d|^2 already formed (r2 unused by FD).
template <int MODE, bool EW, bool ENERGY = false>
__device__ __forceinline__ void pair_two_d(const Cst<float>& k, const PairK2& c, const float2 (&d)[3], float2 r2,
                                           float rc2e, const float2 (&ei)[3], const float2 (&ej)[3], float2 (&a)[3],
                                           float2 (&f)[3], const PairK<float>* ce = nullptr, float ew = 0.f,
                                           float* e = nullptr, float2 eps2 = float2{0.f, 0.f}) {
  if constexpr (MODE == 2) {
    // F(+) - F(-) at the pair separated by d +- eps (e_i - e_j), both beads at once
    const float2 u[3] = {mul2(eps2, sub2(ei[0], ej[0])), mul2(eps2, sub2(ei[1], ej[1])), mul2(eps2, sub2(ei[2], ej[2]))};
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      const float2 q[3] = {sgn ? sub2(d[0], u[0]) : add2(d[0], u[0]), sgn ? sub2(d[1], u[1]) : add2(d[1], u[1]),
                           sgn ? sub2(d[2], u[2]) : add2(d[2], u[2])};
      const float2 r2 = fma2(q[0], q[0], fma2(q[1], q[1], mul2(q[2], q[2])));
      const bool in0 = r2.x < rc2e, in1 = r2.y < rc2e;
      const float2 rinv = rsq2(r2);
      const float2 rinv2 = mul2(rinv, rinv);
      const float2 rinv6 = mul2(mul2(rinv2, rinv2), rinv2);
      const float2 lj = mul2(rinv6, fma2(c.A, rinv6, c.nB));
      float2 g;
      if (EW) {
        float2 ec, c2e;
        ewald_terms2(k, r2, rinv, &ec, &c2e);
        g = fma2(rinv2, fma2(c.qq, fma2(ec, rinv, c2e), lj), mul2(c.sh, rinv));
      } else {
        g = fma2(rinv2, fma2(c.qq, rinv, lj), fma2(c.sh, rinv, c.nqk));
      }
      g = make_float2(in0 ? (sgn ? -g.x : g.x) : 0.f, in1 ? (sgn ? -g.y : g.y) : 0.f);
#pragma unroll
      for (int t = 0; t < 3; ++t) f[t] = sgn ? fma2(g, q[t], f[t]) : mul2(g, q[t]);
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) a[t] = add2(a[t], f[t]);
    return;
  }
  const bool in0 = r2.x < rc2e, in1 = r2.y < rc2e;
  const float2 rinv = rsq2(r2);
  const float2 rinv2 = mul2(rinv, rinv);
  const float2 rinv6 = mul2(mul2(rinv2, rinv2), rinv2);
  const float2 lj = mul2(rinv6, fma2(c.A, rinv6, c.nB));   // r^-6 (A r^-6 - B)
  float2 g, ec, c2e;
  if (EW) {
    ewald_terms2(k, r2, rinv, &ec, &c2e);
    g = fma2(rinv2, fma2(c.qq, fma2(ec, rinv, c2e), lj), mul2(c.sh, rinv));
  } else {
    g = fma2(rinv2, fma2(c.qq, rinv, lj), fma2(c.sh, rinv, c.nqk));
  }
  if (MODE == 0) {
    g = make_float2(in0 ? g.x : 0.f, in1 ? g.y : 0.f);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      f[q] = mul2(g, d[q]);
      a[q] = add2(a[q], f[q]);
    }
    if (ENERGY) {
      // phi(r) - phi(rc) - (r - rc) phi'(rc) of bead x
      const float r = r2.x * rinv.x;
      const float elj = rinv6.x * fmaf(ce->A * (1.f / 12.f), rinv6.x, -ce->B * (1.f / 6.f));
      const float el = EW ? ce->qq * fmaf(ec.x, rinv.x, -k.ewec) : ce->qq * (rinv.x + fmaf(k.krf, r2.x, -k.crf));
      const float E = elj + el - ce->Ew - (r - k.rc) * ce->sh;
      *e = in0 ? fmaf(ew, E, *e) : *e;
    }
  } else {
    const float2 u[3] = {sub2(ei[0], ej[0]), sub2(ei[1], ej[1]), sub2(ei[2], ej[2])};
    const float2 rinv3 = mul2(rinv, rinv2);
    const float2 ljb = mul2(mul2(rinv2, rinv2), mul2(rinv6, fma2(c.A14, rinv6, c.nB8)));
    float2 b;
    if (EW) {
      // r^-3 [qq (3 ec r^-2 + c2E (3 r^-1 + 2 beta^2 r)) + sh]
      const float2 el = fma2(mul2(dup2(3.f), ec), rinv2,
                             mul2(c2e, fma2(dup2(2.f * k.ewb2), mul2(r2, rinv), mul2(dup2(3.f), rinv))));
      b = fma2(rinv3, fma2(c.qq, el, c.sh), ljb);
    } else {
      b = fma2(rinv3, fma2(c.q3, rinv2, c.sh), ljb);
    }
    const float2 sdot = fma2(d[0], u[0], fma2(d[1], u[1], mul2(d[2], u[2])));
    float2 t = mul2(b, sdot);
    t = make_float2(in0 ? t.x : 0.f, in1 ? t.y : 0.f);
    const float2 ng = make_float2(in0 ? -g.x : 0.f, in1 ? -g.y : 0.f);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      f[q] = fma2(ng, u[q], mul2(t, d[q]));
      a[q] = add2(a[q], f[q]);
    }
  }
}

template <int MODE, bool EW, bool ENERGY = false>
__device__ __forceinline__ void pair_two(const Cst<float>& k, const PairK2& c, const float2 (&xs)[3], const float2 (&xj)[3],
                                         float rc2e, const float2 (&ei)[3], const float2 (&ej)[3], float2 (&a)[3],
                                         float2 (&f)[3], const PairK<float>* ce = nullptr, float ew = 0.f,
                                         float* e = nullptr, float2 eps2 = float2{0.f, 0.f}) {
  const float2 d[3] = {sub2(xs[0], xj[0]), sub2(xs[1], xj[1]), sub2(xs[2], xj[2])};
  const float2 r2 = MODE == 2 ? float2{0.f, 0.f} : fma2(d[0], d[0], fma2(d[1], d[1], mul2(d[2], d[2])));
  pair_two_d<MODE, EW, ENERGY>(k, c, d, r2, rc2e, ei, ej, a, f, ce, ew, e, eps2);
}

// j-partial staging of one entry: value (h, c, b) of i-lane ii and j-atom jq at
// ii * kJpRow + jq * 6 + h * 24 + 2c + b.  Both the 64-bit stores (16 lanes per phase: 8 ii x
// 2 jq) and the 64-bit loads of the 24 summing lanes then hit every bank once per phase.
constexpr int kJpRow = 52;
// entries whose j-side partials are staged before one flush (divides the 4 entries of a block;
// more would take the warp staging past the static shared-memory limit)
#ifndef MOP_JBATCH
#define MOP_JBATCH 2
#endif
constexpr int kJBatch = MOP_JBATCH;
// unrolling of the 4-entry loop of a staged block
#ifndef MOP_Q_UNROLL
#define MOP_Q_UNROLL 4
#endif
constexpr int kQUnroll = MOP_Q_UNROLL;

// Warp-private staging area: one chunk of up to 32 list entries, the 32 j-atoms (4 entries x 8
// atoms) of the block being processed for each of the B beads, and the double-float partial
// sums (hi, lo) of every lane.
template <class R, int B> struct Stage {
  using V4 = typename Tr<R>::V4;
  V4 x[B][32];                  // j coordinates + charge (interleaved layout: x x' y y', z z' q type)
  V4 e[B][32];                  // j eta (HVP / FD)
  V4 d[32];                     // Delta of each staged entry (FP64; FP32 reads it from the entry)
  int4 ent[2][32];              // entries of the chunk (force kernels: two buffers, the next in flight)
  unsigned long long m[2][32];  // exclusion masks of the chunk
  int t[32];                    // j types (layouts without the type in x)
  R hl[B][6][32];            // folded sums: hi x 3, lo x 3 (FP32 mode)
  // half list (FP32 mode): j-side partials of kJBatch entries
  float jp[kJBatch][kCL * kJpRow];
  // FP32 HVP and FD units: the j fetch's base pointers (coordinates and eta of the unit's first
  // bead, types), kept here instead of in registers
  const float4* fxq;
  const float4* feta;
  const int* fts;
};

template <class R, class V4>
__device__ __forceinline__ V4 load_eta4(const PathDev& P, size_t k);
template <> __device__ __forceinline__ float4 load_eta4<float, float4>(const PathDev& P, size_t k) {
  return __ldg(&P.eta32[k]);
}
template <> __device__ __forceinline__ double4_32a load_eta4<double, double4_32a>(const PathDev& P, size_t k) {
  return make_double4_32a(P.eta[3 * k], P.eta[3 * k + 1], P.eta[3 * k + 2], 0.0);
}

// fold the FP32 chunk sums a[b][3] of this lane into its (hi, lo) pairs in shared memory
template <class R, int B>
__device__ __forceinline__ void fold_into(Stage<R, B>& S, R (&a)[B][3], int lane) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float h = S.hl[b][c][lane], l = S.hl[b][3 + c][lane];
        two_sum_add(h, l, a[b][c]);
        S.hl[b][c][lane] = h;
        S.hl[b][3 + c][lane] = l;
        a[b][c] = 0.f;
      }
  }
}

// round(s * kFixScale) as int64 (saturating beyond 2^40 in magnitude).  One conversion; the
// FP32-only splits measured slower in this latency-bound loop.
__device__ __forceinline__ unsigned long long to_fix(float s) {
  return (unsigned long long)__float2ll_rn(s * kFixScale);
}

// cp.async (sm_80+): global -> shared copies that bypass registers; waited with wait_group 0
#ifndef MOP_ASYNC_ENT
#define MOP_ASYNC_ENT 1
#endif
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Per-lane constants of the half-list j-side flush, fixed for a whole unit.
struct JFlush {
  int w;         // float offset of this lane's 12 j-partials in a staging slot
  int r;         // reading lanes: float offset of the column this lane sums
  int o1;        // offset of the second bead's j-side sums from the first's
  int oc;        // offset of j-atom a, component c within a j-cluster's 24 sums
  int hbit;      // half-mask bit of the j-atom this lane reads (0: lane does not read)
  bool second;   // the unit's second bead is real
};

// Stores this lane's j-side contributions of one entry: jf[h][c][b] belongs to j-atom
// (lane >> 3) + 4h, component c, bead b (unpacked units; packed units store each active half
// right after its pair evaluation).
template <int B>
__device__ __forceinline__ void j_stage(float* slot, const JFlush& J, const float (&jf)[2][3][B]) {
  static_assert(B == 2, "the j-partial layout holds two beads");
  float2* w = reinterpret_cast<float2*>(slot + J.w);
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int c = 0; c < 3; ++c) w[h * 12 + c] = make_float2(jf[h][c][0], jf[h][c][1]);
}

// Half list: sums the staged j-side contributions of kJBatch entries (the first is entry e0 of
// the chunk) over the 8 i-lanes in a fixed order and adds them, fixed point, to each
// j-cluster's atoms of both beads.  Lane < 24 reads j-atom a = lane / 3, component lane % 3.
// The self entry, entries past the end of the chunk and halves whose bit is clear (not listed, or
// skipped by the vote) add nothing.  jscale[b] maps a sum to the value added (sign and FD scale).
template <int B>
__device__ __forceinline__ void j_flush(const JFlush& J, Stage<float, B>& S, int cb, int e0, unsigned long long* jacc,
                                        const float* jscale) {
  __syncwarp();
#pragma unroll
  for (int q = 0; q < kJBatch; ++q) {
    const int fl = S.ent[cb][e0 + q].x;
    if ((fl & J.hbit) && !(fl & kSelfFlag)) {
      const float* r = &S.jp[q][J.r];
      float2 t[kCL];
#pragma unroll
      for (int ii = 0; ii < kCL; ++ii) t[ii] = *reinterpret_cast<const float2*>(r + ii * kJpRow);
      const float s0 = ((t[0].x + t[1].x) + (t[2].x + t[3].x)) + ((t[4].x + t[5].x) + (t[6].x + t[7].x));
      const float s1 = ((t[0].y + t[1].y) + (t[2].y + t[3].y)) + ((t[4].y + t[5].y) + (t[6].y + t[7].y));
      unsigned long long* dst = jacc + (size_t)(fl & kCluMask) * (kCL * 3) + J.oc;
      atomicAdd(dst, to_fix(s0 * jscale[0]));
      if (J.second) atomicAdd(dst + J.o1, to_fix(s1 * jscale[1]));
    }
  }
  __syncwarp();
}

// One work unit: the i-cluster ci against its whole list, for the B beads n0 .. n0 + B - 1
// (bead n0 + 1 of a unit past the last bead repeats bead n0 and is not written).  FP32 mode runs
// on the half list (each cluster pair once, j-side sums to P.jacc), FP64 mode on the full list.
template <class R, int MODE, bool ENERGY, int B, bool EW>
__device__ __forceinline__ void pair_unit(const SysConsts& sc, const typename Tr<R>::V4* __restrict__ tab, int tstr,
                                          Stage<R, B>& S, const PathDev& P, int n0, int n_pass, int ci, int lane) {
  using V4 = typename Tr<R>::V4;
  constexpr bool HALF = sizeof(R) == 4;
  static_assert(!HALF || B == 2, "the half-list flush pairs two beads");
  const Cst<R> k(sc);
  const int i = lane & 7, jj = lane >> 3;
  const int si = ci * kCL + i;
  int nb[B];
  bool bval[B];
  V4 xi[B];
  R ei[B][3], eps[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    bval[b] = n0 + b < n_pass;
    nb[b] = min(n0 + b, n_pass - 1);
    xi[b] = Tr<R>::xq(P)[(size_t)nb[b] * P.Qpad + si];
    ei[b][0] = ei[b][1] = ei[b][2] = R(0);
    eps[b] = R(0);
    if (MODE >= 1) Tr<R>::eta(P, (size_t)nb[b] * P.Qpad + si, ei[b]);
    if (MODE == 2) {
      const float mx = __uint_as_float(P.etamax[nb[b]]);
      eps[b] = (R)(mx > 0.f ? sc.fd_h / (double)mx : sc.fd_h);
    }
  }
  // slot offset of the unit's first bead, and of its last bead from the first
  const size_t eos0 = (size_t)nb[0] * P.Qpad;
  const int edb = (nb[B - 1] - nb[0]) * P.Qpad;
  // half list: j-side flush constants; atom j gets -f, or +f / (2 eps) in FD mode
  float jscale[B];
#pragma unroll
  for (int b = 0; b < B; ++b) jscale[b] = (MODE == 2) ? 0.5f / (float)eps[b] : -1.f;
  JFlush J{};
  unsigned long long* jacc = nullptr;
  if constexpr (HALF) {
    const int ra = lane / 3, rc = lane - 3 * ra;   // reading lane: j-atom of the entry, component
    J.w = i * kJpRow + jj * 6;
    J.r = (ra & 3) * 6 + (ra >> 2) * 24 + rc * 2;
    J.hbit = lane < 24 ? 1 << (29 + (ra >> 2)) : 0;
    J.oc = ra * 3 + rc;
    J.o1 = (nb[B - 1] - nb[0]) * P.Qpad * 3;
    J.second = bval[B - 1] && B > 1;
    jacc = P.jacc + (size_t)nb[0] * P.Qpad * 3;
  }
  const V4* __restrict__ tabrow = tab + __ldg(&P.ts[si]) * tstr;
  const R qi = xi[0].w;
  // both beads in f32x2 instructions (forces with the bead-1 energy in the first units, the
  // adjoint HVP and the FD difference)
  constexpr bool PACK = MOP_PACK2 && sizeof(R) == 4 && B == 2;
  // interleaved j staging (with the j type in it): measured faster for every packed kernel once
  // their registers were trimmed (reaction-field H eta 15.44 -> 15.10 ms, force -0.15 ms, Ewald
  // -0.2 ms per pass on the 150k-atom path)
  constexpr bool ILV = PACK && MOP_ILV;
  // half skipping by warp vote (measured faster for every packed kernel)
  constexpr bool SKIP = PACK && MOP_SKIP;
  // FD pairs sit at d +- u with |u| = eps |eta_i - eta_j| <= 2 h (eps = h / max |eta|): a half
  // with no |d| < rc + 2 h in either bead holds no pair the FD difference can see
  const float rskip2 = MODE == 2 ? (float)((sc.rc + 2.0 * sc.fd_h) * (sc.rc + 2.0 * sc.fd_h)) : 0.f;
  float2 a2[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  float2 ei2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) ei2[c] = make_float2((float)ei[0][c], (float)ei[B - 1][c]);

  R a[B][3];
  // packed partial sums -> a[b][c] (zero between folds) before each fold
  auto unpack = [&]() __attribute__((always_inline)) {
    if constexpr (PACK) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a[0][c] = a2[c].x;
        a[B - 1][c] = a2[c].y;
        a2[c] = make_float2(0.f, 0.f);
      }
    }
  };
  Acc3<R> accd;   // FP64 mode accumulates directly (B == 1)
#pragma unroll
  for (int b = 0; b < B; ++b) a[b][0] = a[b][1] = a[b][2] = R(0);
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int c = 0; c < 6; ++c) S.hl[b][c][lane] = 0.f;
  }
  Acc1<R> eacc;
  // HVP and FD kernels (FP32): the j fetch's base pointers live in shared memory, freeing
  // registers (spill 24 -> 8 B, H eta 16.68 -> 16.60 ms on the 150k-atom path); the force
  // kernels measured slower that way (13.01 -> 13.33 ms) and keep them in registers
  constexpr bool SPTR = sizeof(R) == 4 && MODE >= 1 && MOP_SPTR;
  if constexpr (SPTR) {
    if (lane == 0) {
      S.fxq = P.xq + eos0;
      S.feta = P.eta32 + eos0;
      S.fts = P.ts;
    }
  }
  const int cnt = __ldg(&P.lcnt[ci]);
  const size_t eb = (size_t)ci * P.cap;
  const int mshift = jj * kCL + i;   // exclusion bit of pair (i, jj); pair (i, jj + 4) is 32 higher
  const int sa = lane & 7, sk = lane >> 3;   // staging role: atom sa of block entry sk
  // force kernels: each 32-entry chunk of the list (entries and masks) is copied into shared
  // memory by cp.async while the previous chunk is processed; entries past the list are zero (no
  // bits).  Measured: reaction-field force 12.20 -> 12.05 ms; the H eta kernels lost (+0.08 ms,
  // Ewald +0.94 ms) and load each chunk when they reach it.
  constexpr bool ASYNC = sizeof(R) == 4 && MOP_ASYNC_ENT && MODE == 0;
  auto issue = [&](int c0n, int buf) __attribute__((always_inline)) {
    if (lane < cnt - c0n) {
      cp_async16(&S.ent[buf][lane], &P.ent[eb + c0n + lane]);
      cp_async8(&S.m[buf][lane], &P.emask[eb + c0n + lane]);
    } else {
      S.ent[buf][lane] = make_int4(0, 0, 0, 0);
    }
    cp_async_commit();
  };
  int cb = 0;
  if constexpr (ASYNC) {
    if (cnt > 0) issue(0, 0);
  }
  for (int c0 = 0; c0 < cnt; c0 += 32) {
    const int nc = min(32, cnt - c0);
    __syncwarp();
    if constexpr (ASYNC) {
      cp_async_wait_all();
      __syncwarp();
      if (c0 + 32 < cnt) issue(c0 + 32, cb ^ 1);
    } else {
      int4 en = make_int4(0, 0, 0, 0);
      unsigned long long m = 0ull;
      V4 dv;
      if (lane < nc) {
        en = __ldg(&P.ent[eb + c0 + lane]);
        if (en.x < 0) m = __ldg(&P.emask[eb + c0 + lane]);
        R D[3];
        Tr<R>::delta(P, eb + c0 + lane, en, D);
        dv.x = D[0];
        dv.y = D[1];
        dv.z = D[2];
        dv.w = R(0);
      }
      S.ent[cb][lane] = en;
      S.m[cb][lane] = m;
      if constexpr (sizeof(R) == 8) S.d[lane] = dv;
      __syncwarp();
    }
    V4 fx[B], fe[B];
    int ft = 0;
    // forced inline: as a call, fx and fe would live in local memory
    auto fetch = [&](int blk) __attribute__((always_inline)) {
      const int e = 4 * blk + sk;
      if (e < nc) {
        const int sj = (S.ent[cb][e].x & kCluMask) * kCL + sa;
        if constexpr (SPTR) {
          ft = __ldg(S.fts + sj);
          const float4* xb = S.fxq;
          const float4* eb4 = S.feta;
#pragma unroll
          for (int b = 0; b < B; ++b) {
            fx[b] = __ldg(xb + (b ? edb : 0) + sj);
            if (MODE >= 1) fe[b] = __ldg(eb4 + (b ? edb : 0) + sj);
          }
        } else {
          ft = __ldg(&P.ts[sj]);
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const size_t o = eos0 + (b ? edb : 0) + sj;
            fx[b] = Tr<R>::xq(P)[o];
            if (MODE >= 1) fe[b] = load_eta4<R, V4>(P, o);
          }
        }
      }
    };
    fetch(0);
    const int nblk = (nc + 3) >> 2;
    for (int blk = 0; blk < nblk; ++blk) {
      __syncwarp();
      if constexpr (ILV) {
        // (z, z', q, type): the packed kernels read the j type from here, not from S.t
        S.x[0][lane] = V4{fx[0].x, fx[B - 1].x, fx[0].y, fx[B - 1].y};
        S.x[B - 1][lane] = V4{fx[0].z, fx[B - 1].z, fx[0].w, __int_as_float(ft)};
        if (MODE >= 1) {
          S.e[0][lane] = V4{fe[0].x, fe[B - 1].x, fe[0].y, fe[B - 1].y};
          S.e[B - 1][lane] = V4{fe[0].z, fe[B - 1].z, R(0), R(0)};
        }
      } else {
#pragma unroll
        for (int b = 0; b < B; ++b) {
          S.x[b][lane] = fx[b];
          if (MODE >= 1) S.e[b][lane] = fe[b];
        }
      }
      if constexpr (!ILV) S.t[lane] = ft;
      __syncwarp();
      if (blk + 1 < nblk) fetch(blk + 1);
      // entries past the end of the chunk were staged with no half bits
#pragma unroll kQUnroll
      for (int q = 0; q < 4; ++q) {
        const int e = 4 * blk + q;
        // FP32: one 128-bit read gives the entry's flags and its Delta (y, z, w)
        const int4 E = S.ent[cb][e];
        const int fl = E.x;
        R rcA = k.rc2, rcB = k.rc2;
        if (fl < 0) {
          const unsigned long long m = S.m[cb][e] >> mshift;
          rcA = (m & 1ull) ? R(-1) : k.rc2;
          rcB = ((m >> 32) & 1ull) ? R(-1) : k.rc2;
        }
        V4 D;
        if constexpr (sizeof(R) == 4) {
          D.x = __int_as_float(E.y);
          D.y = __int_as_float(E.z);
          D.z = __int_as_float(E.w);
        } else {
          D = S.d[e];
        }
        const int so = q * kCL + jj;
        const R ew = (fl & kSelfFlag) ? R(0.5) : R(1);   // the self entry sees each pair twice
        R jf[2][3][B];
        if constexpr (!PACK) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int b = 0; b < B; ++b) jf[h][c][b] = R(0);
        }
        R xs[B][3];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          xs[b][0] = xi[b].x + D.x;
          xs[b][1] = xi[b].y + D.y;
          xs[b][2] = xi[b].z + D.z;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!(fl & (1 << (29 + h)))) continue;
          const int sj = so + 4 * h;
          const R qj = ILV ? S.x[B - 1][sj].z : S.x[0][sj].w;
          const R rce = h ? rcB : rcA;
          // the type-pair row is read before the skip vote: read after it, its latency showed
          // (reaction-field force 12.27 -> 12.66 ms, H eta 15.42 -> 15.70 ms)
          // interleaved staging carries the j type in (z, z', q, type)
          const V4 tp = tabrow[ILV ? __float_as_int(S.x[B - 1][sj].w) : S.t[sj]];
          if constexpr (PACK) {
            const float2 xs2[3] = {make_float2(xs[0][0], xs[B - 1][0]), make_float2(xs[0][1], xs[B - 1][1]),
                                   make_float2(xs[0][2], xs[B - 1][2])};
            const V4 xj0 = S.x[0][sj], xj1 = S.x[B - 1][sj];
            float2 xj2[3], ej2[3];
            if constexpr (ILV) {
              xj2[0] = make_float2(xj0.x, xj0.y);
              xj2[1] = make_float2(xj0.z, xj0.w);
              xj2[2] = make_float2(xj1.x, xj1.y);
            } else {
              xj2[0] = make_float2(xj0.x, xj1.x);
              xj2[1] = make_float2(xj0.y, xj1.y);
              xj2[2] = make_float2(xj0.z, xj1.z);
            }
            // the j-atom's eta (HVP, FD), read after the skip vote
            auto load_ej = [&]() __attribute__((always_inline)) {
              const V4 ej0 = MODE >= 1 ? S.e[0][sj] : V4{}, ej1 = MODE >= 1 ? S.e[B - 1][sj] : V4{};
              if constexpr (ILV) {
                ej2[0] = make_float2(ej0.x, ej0.y);
                ej2[1] = make_float2(ej0.z, ej0.w);
                ej2[2] = make_float2(ej1.x, ej1.y);
              } else {
                ej2[0] = make_float2(ej0.x, ej1.x);
                ej2[1] = make_float2(ej0.y, ej1.y);
                ej2[2] = make_float2(ej0.z, ej1.z);
              }
            };
            constexpr bool EJL = MOP_EJ_LATE && MODE == 1;
            if constexpr (!EJL) load_ej();
            // separation and squared distance of both beads, shared by the skip vote and the pair
            const float2 dd[3] = {sub2(xs2[0], xj2[0]), sub2(xs2[1], xj2[1]), sub2(xs2[2], xj2[2])};
            const float2 r2 = fma2(dd[0], dd[0], fma2(dd[1], dd[1], mul2(dd[2], dd[2])));
            if constexpr (SKIP) {
              // the list holds this half for some bead of the path; when no lane has a pair
              // within rc in either bead of the unit, the warp skips it and clears its bit, so
              // that the flush does not read the row either
              const float rv = MODE == 2 ? (rce > 0.f ? rskip2 : -1.f) : rce;
              if (!__any_sync(0xffffffffu, r2.x < rv || r2.y < rv)) {
                if (lane == 0) S.ent[cb][e].x &= ~(1 << (29 + h));
                continue;
              }
            }
            if constexpr (EJL) load_ej();
            const PairK<R> pc = pair_consts<R, MODE, V4>(k, tp, qi * qj);
            float2 f2[3];
            pair_two_d<MODE, EW, ENERGY>(k, pair_consts2<MODE>(pc), dd, r2, rce, ei2, ej2, a2, f2, &pc, ew, &eacc.a,
                                         make_float2((float)eps[0], (float)eps[B - 1]));
            // straight to this lane's staging row; the row of a half without its bit is never read
            float2* w = reinterpret_cast<float2*>(S.jp[q % kJBatch] + J.w) + h * 12;
#pragma unroll
            for (int c = 0; c < 3; ++c) w[c] = f2[c];
            continue;
          }
          const PairK<R> pc = pair_consts<R, MODE, V4>(k, tp, qi * qj);
#pragma unroll
          for (int b = 0; b < B; ++b) {
            R ej[3] = {R(0), R(0), R(0)};
            if (MODE >= 1) {
              const V4 v = S.e[b][sj];
              ej[0] = v.x;
              ej[1] = v.y;
              ej[2] = v.z;
            }
            R* acc = (sizeof(R) == 4) ? a[b] : accd.a;
            R f[3];
            if (ENERGY && b == 0)   // energy of bead n0 (= bead 1) only
              pair_one<R, MODE, true, HALF, EW, V4>(k, pc, xs[b][0], xs[b][1], xs[b][2], S.x[b][sj], rce, ei[b], ej,
                                                eps[b], ew, acc, eacc.a, f);
            else
              pair_one<R, MODE, false, HALF, EW, V4>(k, pc, xs[b][0], xs[b][1], xs[b][2], S.x[b][sj], rce, ei[b], ej,
                                                 eps[b], ew, acc, eacc.a, f);
            if (HALF) {
#pragma unroll
              for (int c = 0; c < 3; ++c) jf[h][c][b] = f[c];
            }
          }
        }
        if constexpr (HALF) {
          if constexpr (!PACK) j_stage<B>(S.jp[q % kJBatch], J, jf);
          if (q % kJBatch == kJBatch - 1) j_flush<B>(J, S, cb, e - (kJBatch - 1), jacc, jscale);
        }
      }
      if ((blk & 3) == 3) {
        unpack();
        fold_into<R, B>(S, a, lane);
        if (ENERGY) eacc.fold();
      }
    }
    if constexpr (ASYNC) cb ^= 1;
  }
  unpack();
  fold_into<R, B>(S, a, lane);
  if (ENERGY) eacc.fold();
  const bool valid = __ldg(&P.perm[si]) >= 0;
  if constexpr (sizeof(R) == 4) {
    // sum the four lanes of each i-atom as double-floats, no FP64 instructions
#pragma unroll
    for (int b = 0; b < B; ++b) {
      df v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[c] = df{S.hl[b][c][lane], S.hl[b][3 + c][lane]};
#pragma unroll
        for (int o = 8; o <= 16; o <<= 1) {
          const df w{__shfl_xor_sync(0xffffffffu, v[c].hi, o), __shfl_xor_sync(0xffffffffu, v[c].lo, o)};
          v[c] = df_add(v[c], w);
        }
        if (!valid) v[c] = df{0.f, 0.f};
      }
      if (jj == 0 && bval[b]) {
        const size_t k2 = (size_t)nb[b] * P.Qpad + si;
        if (MODE == 0) {
          float2* dst = reinterpret_cast<float2*>(P.Fnb) + 3 * k2;
          dst[0] = make_float2(v[0].hi, v[0].lo);
          dst[1] = make_float2(v[1].hi, v[1].lo);
          dst[2] = make_float2(v[2].hi, v[2].lo);
        } else {
          const float scale = (MODE == 2) ? -0.5f / (float)eps[b] : 1.0f;
          reinterpret_cast<float4*>(P.Hnb)[k2] = make_float4((v[0].hi + v[0].lo) * scale,
                                                             (v[1].hi + v[1].lo) * scale,
                                                             (v[2].hi + v[2].lo) * scale, 0.f);
        }
      }
    }
    if (ENERGY) {
      df ev = valid ? df{eacc.h, eacc.l} : df{0.f, 0.f};
      ev = df_warp_sum(ev);
      if (lane == 0) P.e_pair[ci] = (double)ev.hi + (double)ev.lo;   // half list: each pair once
    }
  } else {
    double out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double v = accd.get(c);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      out[c] = valid ? v : 0.0;
    }
    if (jj == 0) {
      double* dst = (MODE == 0 ? P.Fnb : P.Hnb) + 3 * ((size_t)nb[0] * P.Qpad + si);
      const double scale = (MODE == 2) ? -0.5 / (double)eps[0] : 1.0;
      dst[0] = out[0] * scale;
      dst[1] = out[1] * scale;
      dst[2] = out[2] * scale;
    }
    if (ENERGY) {
      double ev = valid ? eacc.get() : 0.0;
      ev = warp_sum(ev);
      if (lane == 0) P.e_pair[ci] = 0.5 * ev;   // full list: every pair seen twice
    }
  }
}

template <class R> struct BeadsPerUnit { static constexpr int value = sizeof(R) == 4 ? 2 : 1; };

template <class R, int MODE, bool EW>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? MOP_PAIR_MINB : 2) k_pair(SysConsts sc, const PathDev* __restrict__ paths,
                                                                      int n_paths, long long u_begin, long long n_units) {
  using V4 = typename Tr<R>::V4;
  constexpr int B = BeadsPerUnit<R>::value;
  // type-pair table with an odd row stride: the 8 i-lanes of a quarter-warp (one j type, up to
  // 8 i types) then read distinct banks
  __shared__ V4 tab[kMaxTypes * (kMaxTypes + 1)];
  __shared__ Stage<R, B> stage[4];
  const int tstr = sc.n_types | 1;
  for (int k = threadIdx.x; k < sc.n_types * tstr; k += blockDim.x) {
    const int ti = k / tstr, tj = k - ti * tstr;
    tab[k] = tj < sc.n_types ? Tr<R>::tab(sc, ti * sc.n_types + tj) : V4{};
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  Stage<R, B>& S = stage[threadIdx.x >> 5];
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = u_begin + (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); u < n_units; u += nw) {
    int p = 0;
    if (MODE == 0) {
      while (p + 1 < n_paths && paths[p + 1].unit_off <= u) ++p;
    } else {
      while (p + 1 < n_paths && paths[p + 1].unit_off_h <= u) ++p;
    }
    const PathDev& P = paths[p];
    const int n_pass = MODE == 0 ? P.n_force : P.n_hvp;
    // bead-major: the warps in flight share a few beads, so their coordinates and j-side sums
    // stay in L2
    const long long v = u - (MODE == 0 ? P.unit_off : P.unit_off_h);
    const int n0 = (int)(v / P.n_clu) * B;
    const int ci = (int)(v % P.n_clu);
    if (ci >= __ldg(&P.meta[0])) continue;   // past the clusters of the current sort
    if (MODE == 0 && n0 == 0) pair_unit<R, 0, true, B, EW>(sc, tab, tstr, S, P, n0, n_pass, ci, lane);
    else pair_unit<R, MODE, false, B, EW>(sc, tab, tstr, S, P, n0, n_pass, ci, lane);
  }
}

template <class R, int MODE, bool EW>
cudaError_t launch_one(const SysConsts& sc, const PathDev* d_paths, int n_paths, long long u_begin, long long n_units,
                       int num_sms, Launch L) {
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair<R, MODE, EW>, 128, 0);
    if (e != cudaSuccess || per_sm <= 0) per_sm = 4;
  }
  const long long want_blocks = (n_units - u_begin + 3) / 4;
  long long blocks = (long long)num_sms * per_sm;
  if (blocks > want_blocks) blocks = want_blocks;
  if (blocks < 1) blocks = 1;
  k_pair<R, MODE, EW><<<(int)blocks, 128, 0, L.st>>>(sc, d_paths, n_paths, u_begin, n_units);
  ++*L.counter;
  return cudaGetLastError();
}

// in-cutoff, non-excluded ordered pairs of every force unit, and the pairs the list makes the
// force kernel evaluate (instrumentation)
__global__ void k_count_pairs(SysConsts sc, const PathDev* __restrict__ paths, int n_paths, long long n_units,
                              unsigned long long* counts) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long inside = 0, listed = 0;
  for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n_units; u += nw) {
    int p = 0;
    while (p + 1 < n_paths && paths[p + 1].unit_off <= u) ++p;
    const PathDev& P = paths[p];
    const long long v = u - P.unit_off;
    const int n = (int)(v % P.n_force), ci = (int)(v / P.n_force);
    if (ci >= P.meta[0]) continue;
    const int i = lane & 7, jj = lane >> 3;
    const size_t bo = (size_t)n * P.Qpad;
    const bool vi = P.perm[ci * kCL + i] >= 0;
    const size_t eb = (size_t)ci * P.cap;
    for (int e = 0; e < P.lcnt[ci]; ++e) {
      const int4 en = P.ent[eb + e];
      const unsigned long long m = (en.x < 0 || sc.bl) ? P.emask[eb + e] : 0ull;
      const int cj = en.x & kCluMask;
      double D[3];
      if (P.ent64) {
        D[0] = P.ent64[eb + e].x; D[1] = P.ent64[eb + e].y; D[2] = P.ent64[eb + e].z;
      } else {
        D[0] = __int_as_float(en.y); D[1] = __int_as_float(en.z); D[2] = __int_as_float(en.w);
      }
      for (int h = 0; h < 2; ++h) {
        if (!(en.x & (1 << (29 + h)))) continue;
        const int jl = jj + 4 * h, sj = cj * kCL + jl;
        // bead-lane list: only the entry's candidate pairs are evaluated (none of them excluded)
        if (sc.bl && !((m >> (jl * kCL + i)) & 1ull)) continue;
        double a[3], b[3];
        if (P.xq64) {
          const double4_32a x = P.xq64[bo + ci * kCL + i], y = P.xq64[bo + sj];
          a[0] = x.x; a[1] = x.y; a[2] = x.z; b[0] = y.x; b[1] = y.y; b[2] = y.z;
        } else if (sc.bl && sc.elec != 1) {
          // the bead-lane coordinates (xq holds bead 1 only): bead n at group n / 64, lane n % 32,
          // half (n / 32) % 2
          const size_t gb = ((size_t)(n / kBLBeads) * P.Qpad) * 3 * 32;
          const int l = n & 31, hh = (n >> 5) & 1;
          for (int c = 0; c < 3; ++c) {
            const float2 x = P.xb[gb + ((size_t)(ci * kCL + i) * 3 + c) * 32 + l];
            const float2 y = P.xb[gb + ((size_t)sj * 3 + c) * 32 + l];
            a[c] = hh ? x.y : x.x;
            b[c] = hh ? y.y : y.x;
          }
        } else {
          const float4 x = P.xq[bo + ci * kCL + i], y = P.xq[bo + sj];
          a[0] = x.x; a[1] = x.y; a[2] = x.z; b[0] = y.x; b[1] = y.y; b[2] = y.z;
        }
        double r2 = 0.0;
        for (int c = 0; c < 3; ++c) {
          const double d = a[c] + D[c] - b[c];
          r2 += d * d;
        }
        const bool vj = P.perm[sj] >= 0;
        // a half-list entry holds each unordered pair once, the self entry (and the full list)
        // each pair in both orders
        // (the bead-lane half list holds the self entry's pairs once as well)
        const int wgt = sc.bl == 2 ? 2 : ((P.jacc && !(en.x & kSelfFlag) && !sc.bl) ? 2 : 1);
        listed += 1;
        const bool excluded = !sc.bl && ((m >> (jl * kCL + i)) & 1ull);
        inside += (vi && vj && r2 < sc.rc2 && !excluded) ? wgt : 0;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    inside += __shfl_xor_sync(0xffffffffu, inside, o);
    listed += __shfl_xor_sync(0xffffffffu, listed, o);
  }
  if (lane == 0) {
    atomicAdd(&counts[0], inside);
    atomicAdd(&counts[1], listed);
  }
}

}  // namespace

cudaError_t launch_count_pairs(const SysConsts& sc, const PathDev* d_paths, int n_paths, long long n_units,
                               unsigned long long* counts, int num_sms, Launch L) {
  cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), L.st);
  if (e != cudaSuccess) return e;
  k_count_pairs<<<num_sms * 4, 128, 0, L.st>>>(sc, d_paths, n_paths, n_units, counts);
  ++*L.counter;
  return cudaGetLastError();
}

int pair_beads_per_unit(int precision) { return precision == 1 ? 1 : 2; }

cudaError_t launch_pair(const SysConsts& sc, const PathDev* d_paths, int n_paths, long long n_units, int mode,
                        int num_sms, Launch L, long long u_begin) {
  if (n_units <= u_begin) return cudaSuccess;
  const bool f64 = sc.precision == 1, ew = sc.elec == 1;   // Ewald runs in mixed precision only
  switch (mode) {
    case 0: return f64 ? launch_one<double, 0, false>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L)
                 : ew ? launch_one<float, 0, true>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L)
                      : launch_one<float, 0, false>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L);
    case 1: return f64 ? launch_one<double, 1, false>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L)
                 : ew ? launch_one<float, 1, true>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L)
                      : launch_one<float, 1, false>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L);
    default: return f64 ? launch_one<double, 2, false>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L)
                  : ew ? launch_one<float, 2, true>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L)
                       : launch_one<float, 2, false>(sc, d_paths, n_paths, u_begin, n_units, num_sms, L);
  }
}

}  // namespace mop
