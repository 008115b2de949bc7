// Bead-lane pair kernels of the hot path (mixed precision): the nonbonded force F(R^n), the
// adjoint Hessian-vector product H(R^n) eta^n, and the finite-difference stand-in of Eq. 5,
// F(R + eps eta) - F(R - eps eta).
//
// Paper: the do_force calls of every bead (Sec. 2.1, Fig. 2) carry most of the computational
// effort; the FD term is the last term of Eq. 5.  All beads of a path share one cluster-pair
// list here, so a warp takes one i-cluster (8 atoms) for a group of 64 beads at once: lane l
// holds beads 64 g + l and 64 g + 32 + l as the two halves of f32x2 operands, keeps the 8
// i-atoms of both beads (coordinates, eta and FP32 sums) in registers, and walks the i-cluster's
// list of j-clusters.  Every lane evaluates the same atom pair at the same time, so the choice
// of pairs is warp-uniform: the list entry's 64-bit mask of candidate pairs (the atoms' union
// spheres over all beads come within rc, excluded pairs removed) selects them, with no
// per-bead screening and no divergence.  The list holds every cluster pair from both sides, and
// one entry of each mirror pair carries an owner flag.  Without HALF a kernel walks every entry,
// so an atom's sum is complete in its own warp: no j-side sums and no atomics (the force pass).
// With HALF it walks the owner entries only (each atom pair once; a self entry's pairs j > i),
// and the warp also sums each j-atom's share over its i-atoms and adds it, with the sign
// reversed, to j-side sums; a later pass (k_bl_combine) adds those to the rows (the H eta and FD
// passes, and both passes of a half list, which holds owner entries only).  The force launch over
// the full list ends with one-warp units that sum the bead-1 pair energy U(R^1) (energy1_warp),
// so that they fill its last wave.
//
// The j-side sums are exact and order-independent: a share v (forces in kJ mol^-1 nm^-1; H eta
// scaled per bead by a power of two, see bl_jscale) becomes an integer on a fixed grid, carried as
// two 32-bit parts hi = round(v / kHi) and lo = round((v - kHi hi) kLo) (FP32 magic-number
// roundings, see BLGrid) packed into one 64-bit word hi 2^32 + lo; a 64-bit integer atomic adds
// it.  Integer sums do not depend on the order of the additions, so the result has the same bits
// whatever order the warps run in.  The low 32 bits of a sum hold the sum of the lo parts exactly
// while it stays below 2^31 (|lo| <= 2^21 per share, a few hundred shares per atom-bead), so both
// sums come back and the value is (sum hi) kHi + (sum lo) / kLo: 64-bit fixed point.

#include <algorithm>

#include "mop_host.h"
#include "mop_pairmath.cuh"

namespace mop {
namespace {

// warps per block (force kernel / HVP and FD kernels): consecutive units of one bead group
#ifndef MOP_BL_WARPS_F
#define MOP_BL_WARPS_F 1
#endif
#ifndef MOP_BL_WARPS_H
#define MOP_BL_WARPS_H 1
#endif
template <int MODE> struct BLWarps { static constexpr int value = MODE == 0 ? MOP_BL_WARPS_F : MOP_BL_WARPS_H; };
// unrolling of the walk over an entry's 8 j-atoms (force / HVP and FD, full list / half list):
// full unrolling makes every offset a constant, partial unrolling keeps the hot loop within the
// instruction cache
#ifndef MOP_BL_JU_F
#define MOP_BL_JU_F 8
#endif
#ifndef MOP_BL_JU_H
#define MOP_BL_JU_H 8
#endif
#ifndef MOP_BL_JU_FH
#define MOP_BL_JU_FH 8
#endif
#ifndef MOP_BL_JU_HH
#define MOP_BL_JU_HH 2
#endif
template <int MODE, bool HALF> struct BLJUnroll {
  static constexpr int value = HALF ? (MODE == 0 ? MOP_BL_JU_FH : MOP_BL_JU_HH) : (MODE == 0 ? MOP_BL_JU_F : MOP_BL_JU_H);
};
#ifndef MOP_BL_FOLD
#define MOP_BL_FOLD 16
#endif
constexpr int kBLFold = MOP_BL_FOLD;   // list entries between folds of the FP32 sums
// i-atoms evaluated together under one warp-uniform branch when all of them are candidates of
// the j-atom: their dependency chains interleave (other groups go one candidate at a time)
#ifndef MOP_BL_ILP
#define MOP_BL_ILP 1
#endif
constexpr int kBLIlp = MOP_BL_ILP;
// check build (a second library for the tests, never the product): a lane whose j-side share
// for a bead exceeds what the scale promises (2^24 for H eta, 2^30 for unscaled forces) writes
// NaN into that bead's rows of the unit, so that a violated bound cannot pass unnoticed
// the j-atoms' rows loaded through L2 only (ld.global.cg): a warp reads each row once per entry,
// and the two warps of a cluster rarely share an SM, so L1 would only hold them at the expense
// of the atomics (config 5: force 5.38 -> 5.33 ms, H eta 7.33 -> 7.28 ms)
#ifndef MOP_BL_JCG
#define MOP_BL_JCG 1
#endif
// the force kernel over the full list also runs the bead-1 pair energy, as one-warp units after its
// own (they fill the kernel's last wave instead of a launch of their own; force pass 5.45 -> 5.39 ms
// at config 5)
#ifndef MOP_BL_E1FUSE
#define MOP_BL_E1FUSE 1
#endif
// j-side words formed by one 64-bit subtraction (1; H eta pass 7.39 -> 7.34 ms at config 5) or
// by packing the two 32-bit parts (0)
#ifndef MOP_BL_PACK64
#define MOP_BL_PACK64 1
#endif
#ifndef MOP_BL_JCHECK
#define MOP_BL_JCHECK 0
#endif

// the entry's j-atom charges and types loaded once per entry and shuffled to the j-loop (force
// kernel: 5.69 -> 5.45 ms at config 5), or loaded per j-atom (H eta and FD kernels: faster there)
#ifndef MOP_BL_QTSHFL_F
#define MOP_BL_QTSHFL_F 1
#endif
#ifndef MOP_BL_QTSHFL_H
#define MOP_BL_QTSHFL_H 0
#endif
template <int MODE> struct BLQtShfl { static constexpr bool value = MODE == 0 ? MOP_BL_QTSHFL_F : MOP_BL_QTSHFL_H; };
#ifndef MOP_BL_JSTATIC
#define MOP_BL_JSTATIC 1
#endif
// next j-atom's loads issued before the current one is evaluated (force / HVP and FD kernels)
#ifndef MOP_BL_JPF_F
#define MOP_BL_JPF_F 0
#endif
// L1 prefetch of the next j-atom's rows (prefetch.global.L1, no registers held)
#ifndef MOP_BL_L1PF
#define MOP_BL_L1PF 0
#endif
// L1 prefetch, while an entry is evaluated, of the rows of the next walked entry's candidate
// j-atoms (force / HVP and FD kernels): an entry's 8 j-atoms are 8 consecutive slots, so their
// rows are 6 KB of consecutive 128-byte lines per array, and two warp instructions per array
// cover the lines of every candidate j-atom
#ifndef MOP_BL_EPF_F
#define MOP_BL_EPF_F 0
#endif
#ifndef MOP_BL_EPF_H
#define MOP_BL_EPF_H 0
#endif
template <int MODE> struct BLEpf { static constexpr bool value = MODE == 0 ? MOP_BL_EPF_F : MOP_BL_EPF_H; };
// HVP and FD kernels: the i-atoms' eta in shared memory instead of registers (more warps)
#ifndef MOP_BL_EISH
#define MOP_BL_EISH 0
#endif
#ifndef MOP_BL_JPF_H
#define MOP_BL_JPF_H 0
#endif
// i-atoms a warp holds: the whole cluster (8), or half of it (4), the two halves of a cluster
// then being consecutive warps of a block that walk the same list (fewer registers, more warps)
#ifndef MOP_BL_I
#define MOP_BL_I 4
#endif
constexpr int kBLI = MOP_BL_I;
constexpr int kBLSplit = kCL / kBLI;
static_assert(kCL % kBLI == 0 && kBLI % kBLIlp == 0, "i-atom split");

// Pair constants of i-atom i against j type tj, pre-duplicated for f32x2 operands, at
// pt[(i * kMaxTypes + tj) * rows]: (A, A, -B, -B), (q_i, q_i, phi'_LJ(rc), phi'_LJ(rc)) and,
// for the HVP kernel, (14 A, 14 A, -8 B, -8 B), with A = 12 c12, B = 6 c6 and q_i = sqrt(f) q.
// The i-atom's offset is then a constant of the unrolled loop.
template <int MODE> struct BLRow { static constexpr int value = MODE == 1 ? 3 : 2; };

// Per-warp shared state: the current chunk of 32 list entries, the pair table of the
// i-cluster, and each lane's folded sums.
template <int MODE> struct BLWarp {
  int4 ent[32];
  unsigned long long m[32];
  float4 pt[kBLI * kMaxTypes * BLRow<MODE>::value];
  float2 hl[2 * kBLI * 3][32];   // lane's folded sums: hi at [a * 3 + c], lo at [3 kBLI + a * 3 + c]
  float2 ei[MOP_BL_EISH && MODE >= 1 ? kBLI * 3 : 1][32];   // i-atoms' eta (MOP_BL_EISH)
};

// Constants of one pair (both halves equal) for the f32x2 arithmetic.
struct BLPair {
  float2 A, nB;     // 12 c12, -6 c6
  float2 qq, sh;    // f q_i q_j, phi'(rc) of the pair
};

// Per-kernel constants.
struct BLConst {
  float2 drf, nk2rf;        // phi'_RF(rc) / (f qq), -2 k_rf (reaction field)
  float ewb, ewb2, ewc2;    // Ewald: beta, beta^2, 2 beta / sqrt(pi)
  float2 tew2;              // Ewald: (2 beta^2, 2 beta^2)
};

// g (force factor) of both halves from the powers of 1/r; EW: the Ewald terms come back in ec, c2e
template <bool EW>
__device__ __forceinline__ float2 bl_g(const BLConst& k, const BLPair& c, float2 r2, float2 rinv, float2 rinv2,
                                       float2 rinv6, float2* ec, float2* c2e) {
  const float2 lj = mul2(rinv6, fma2(c.A, rinv6, c.nB));   // r^-6 (A r^-6 - B)
  if constexpr (EW) {
    ewald_terms2(k.ewb, k.ewb2, k.ewc2, r2, rinv, ec, c2e);
    return fma2(rinv2, fma2(c.qq, fma2(*ec, rinv, *c2e), lj), mul2(c.sh, rinv));
  } else {
    return fma2(rinv2, fma2(c.qq, rinv, lj), fma2(c.sh, rinv, mul2(c.qq, k.nk2rf)));
  }
}

// zero the half of v whose r2 is not below rc2
__device__ __forceinline__ float2 cut2(float2 v, float2 r2, float rc2) {
  return make_float2(r2.x < rc2 ? v.x : 0.f, r2.y < rc2 ? v.y : 0.f);
}

// MODE 0: acc += g d.  d = x_i - (x_j - Delta).  HALF: fj += g d as well (the j-atom's share,
// negated when it is stored)
template <bool EW, bool HALF>
__device__ __forceinline__ void bl_force(const BLConst& k, const BLPair& c, float rc2, const float2 (&xi)[3],
                                         const float2 (&xj)[3], float2 (&acc)[3], float2 (&fj)[3], float2& gm) {
  const float2 d[3] = {sub2(xi[0], xj[0]), sub2(xi[1], xj[1]), sub2(xi[2], xj[2])};
  const float2 r2 = fma2(d[0], d[0], fma2(d[1], d[1], mul2(d[2], d[2])));
  const float2 rinv = rsq2(r2);
  const float2 rinv2 = mul2(rinv, rinv);
  const float2 rinv6 = mul2(mul2(rinv2, rinv2), rinv2);
  float2 ec, c2e;
  const float2 g = cut2(bl_g<EW>(k, c, r2, rinv, rinv2, rinv6, &ec, &c2e), r2, rc2);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    acc[q] = fma2(g, d[q], acc[q]);
    if constexpr (HALF) fj[q] = fma2(g, d[q], fj[q]);
  }
  gm = make_float2(fmaxf(gm.x, fabsf(g.x)), fmaxf(gm.y, fabsf(g.y)));
}

// MODE 1: acc += b (d.u) d - g u with u = eta_i - eta_j.  A14B8 = (14 A, 14 A, -8 B, -8 B).
template <bool EW, bool HALF>
__device__ __forceinline__ void bl_hvp(const BLConst& k, const BLPair& c, float rc2, float4 A14B8, const float2 (&xi)[3],
                                       const float2 (&xj)[3], const float2 (&ei)[3], const float2 (&ej)[3],
                                       float2 (&acc)[3], float2 (&fj)[3]) {
  const float2 d[3] = {sub2(xi[0], xj[0]), sub2(xi[1], xj[1]), sub2(xi[2], xj[2])};
  const float2 r2 = fma2(d[0], d[0], fma2(d[1], d[1], mul2(d[2], d[2])));
  const float2 u[3] = {sub2(ei[0], ej[0]), sub2(ei[1], ej[1]), sub2(ei[2], ej[2])};
  const float2 rinv = rsq2(r2);
  const float2 rinv2 = mul2(rinv, rinv);
  const float2 rinv4 = mul2(rinv2, rinv2);
  const float2 rinv6 = mul2(rinv4, rinv2);
  const float2 rinv3 = mul2(rinv, rinv2);
  float2 ec, c2e;
  const float2 g = bl_g<EW>(k, c, r2, rinv, rinv2, rinv6, &ec, &c2e);
  // LJ part of b: r^-4 r^-6 (14 A r^-6 - 8 B)
  const float2 ljb = mul2(rinv4, mul2(rinv6, fma2(make_float2(A14B8.x, A14B8.y), rinv6, make_float2(A14B8.z, A14B8.w))));
  float2 b;
  if constexpr (EW) {
    // r^-3 [qq (3 ec r^-2 + c2E (3 r^-1 + 2 beta^2 r)) + sh]
    const float2 three = dup2(3.f);
    const float2 el = fma2(mul2(three, ec), rinv2, mul2(c2e, fma2(k.tew2, mul2(r2, rinv), mul2(three, rinv))));
    b = fma2(rinv3, fma2(c.qq, el, c.sh), ljb);
  } else {
    // r^-3 (3 qq r^-2 + sh)
    b = fma2(rinv3, fma2(mul2(dup2(3.f), c.qq), rinv2, c.sh), ljb);
  }
  const float2 s = fma2(d[0], u[0], fma2(d[1], u[1], mul2(d[2], u[2])));
  const float2 t = cut2(mul2(b, s), r2, rc2);
  const float2 ng = cut2(make_float2(-g.x, -g.y), r2, rc2);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    acc[q] = fma2(ng, u[q], fma2(t, d[q], acc[q]));
    if constexpr (HALF) fj[q] = fma2(ng, u[q], fma2(t, d[q], fj[q]));
  }
}

// MODE 2: acc += F_pair(d + eps u) - F_pair(d - eps u), eps per half (bead)
template <bool EW, bool HALF>
__device__ __forceinline__ void bl_fd(const BLConst& k, const BLPair& c, float rc2, float2 eps2, const float2 (&xi)[3],
                                      const float2 (&xj)[3], const float2 (&ei)[3], const float2 (&ej)[3],
                                      float2 (&acc)[3], float2 (&fj)[3]) {
  const float2 d[3] = {sub2(xi[0], xj[0]), sub2(xi[1], xj[1]), sub2(xi[2], xj[2])};
  const float2 u[3] = {mul2(eps2, sub2(ei[0], ej[0])), mul2(eps2, sub2(ei[1], ej[1])),
                       mul2(eps2, sub2(ei[2], ej[2]))};
#pragma unroll
  for (int sgn = 0; sgn < 2; ++sgn) {
    const float2 p[3] = {sgn ? sub2(d[0], u[0]) : add2(d[0], u[0]), sgn ? sub2(d[1], u[1]) : add2(d[1], u[1]),
                         sgn ? sub2(d[2], u[2]) : add2(d[2], u[2])};
    const float2 r2 = fma2(p[0], p[0], fma2(p[1], p[1], mul2(p[2], p[2])));
    const float2 rinv = rsq2(r2);
    const float2 rinv2 = mul2(rinv, rinv);
    const float2 rinv6 = mul2(mul2(rinv2, rinv2), rinv2);
    float2 ec, c2e;
    float2 g = cut2(bl_g<EW>(k, c, r2, rinv, rinv2, rinv6, &ec, &c2e), r2, rc2);
    if (sgn) g = make_float2(-g.x, -g.y);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      acc[q] = fma2(g, p[q], acc[q]);
      if constexpr (HALF) fj[q] = fma2(g, p[q], fj[q]);
    }
  }
}

// (hi, lo) += a for both halves, without loss (Knuth's TwoSum in f32x2)
__device__ __forceinline__ void two_sum_add2(float2& hi, float2& lo, float2 a) {
  const float2 s = add2(hi, a);
  const float2 bp = sub2(s, hi);
  const float2 err = add2(sub2(hi, sub2(s, bp)), sub2(a, bp));
  hi = s;
  lo = add2(lo, err);
}

template <class W>
__device__ __forceinline__ void bl_fold(W& S, float2 (&acc)[kBLI][3], int lane) {
#pragma unroll
  for (int a = 0; a < kBLI; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 h = S.hl[a * 3 + c][lane], l = S.hl[3 * kBLI + a * 3 + c][lane];
      two_sum_add2(h, l, acc[a][c]);
      S.hl[a * 3 + c][lane] = h;
      S.hl[3 * kBLI + a * 3 + c][lane] = l;
      acc[a][c] = make_float2(0.f, 0.f);
    }
}

// x + 1.5 * 2^23 rounds |x| < 2^22 to an integer whose two's complement is the low bits of the
// sum's bit pattern minus that of 1.5 * 2^23
constexpr float kMagic = 12582912.f;
constexpr int kMagicBits = 0x4B400000;

#if !MOP_BL_PACK64
// hi 2^32 + lo as a 64-bit two's complement word: a negative lo borrows one from hi
__device__ __forceinline__ unsigned long long bl_pack(int hi, int lo) {
  return ((unsigned long long)(unsigned)(hi + (lo >> 31)) << 32) | (unsigned)lo;
}
#endif

// Grids of the j-side words: a share v is clamped to |v| <= kMax, hi = round(v / kHi) and
// lo = round((v - kHi hi) kLo), so |lo| <= kHi kLo / 2 = 2^21 and the magic-number roundings
// stay exact.  Force shares (kJ mol^-1 nm^-1, unscaled): kHi = 2^10, kLo = 2^12, |v| <= 2^31;
// H eta shares (scaled to at most 2^24): kHi = 2^4, kLo = 2^18, |v| <= 2^25.
template <int MODE> struct BLGrid {
  static constexpr float kHi = MODE == 0 ? 1024.f : 16.f;
  static constexpr float kLo = MODE == 0 ? 4096.f : 262144.f;
  static constexpr float kMax = MODE == 0 ? 2147483648.f : 33554432.f;
};

// the 64-bit fixed-point words (hi 2^32 + lo) of the shares v of the lane's two beads
template <int MODE>
__device__ __forceinline__ void bl_fix(float2 v, unsigned long long& w0, unsigned long long& w1) {
  using Gd = BLGrid<MODE>;
  v = make_float2(fminf(fmaxf(v.x, -Gd::kMax), Gd::kMax), fminf(fmaxf(v.y, -Gd::kMax), Gd::kMax));
  const float2 t = fma2(v, dup2(1.f / Gd::kHi), dup2(kMagic));   // v / kHi rounded
  const float2 hf = sub2(t, dup2(kMagic));                        // that integer, exactly
  const float2 r = fma2(hf, dup2(-Gd::kHi), v);                   // v - kHi hi, exact
  const float2 u = fma2(r, dup2(Gd::kLo), dup2(kMagic));          // r kLo rounded
#if MOP_BL_PACK64
  // (t 2^32 + u) - M (2^32 + 1) = (t - M) 2^32 + (u - M): the same word as bl_pack, formed by one
  // 64-bit subtraction (the borrow of a negative lo is the subtraction's own)
  constexpr unsigned long long kMM = ((unsigned long long)(unsigned)kMagicBits << 32) | (unsigned)kMagicBits;
  w0 = (((unsigned long long)__float_as_uint(t.x) << 32) | __float_as_uint(u.x)) - kMM;
  w1 = (((unsigned long long)__float_as_uint(t.y) << 32) | __float_as_uint(u.y)) - kMM;
#else
  w0 = bl_pack(__float_as_int(t.x) - kMagicBits, __float_as_int(u.x) - kMagicBits);
  w1 = bl_pack(__float_as_int(t.y) - kMagicBits, __float_as_int(u.y) - kMagicBits);
#endif
}

// value of a sum of such words: (sum hi) kHi + (sum lo) / kLo
template <int MODE>
__device__ __forceinline__ double bl_unfix(unsigned long long w) {
  const long long W = (long long)w;
  const int lo = (int)(unsigned)(w & 0xffffffffull);
  const long long hi = (W - (long long)lo) >> 32;
  return (double)hi * (double)BLGrid<MODE>::kHi + (double)lo * (1.0 / (double)BLGrid<MODE>::kLo);
}

// Power-of-two scale of a bead's j-side shares in the H eta pass (forces use 1).  A share sums at
// most 4 pairs' (|b| r^2 + |g|) |u|, with |u| <= 2 max_i |eta_i| and |b| r^2 <= 14 |g| where the
// repulsion dominates (the LJ and Coulomb parts of b r^2 are 14 and 3 times those of g; near the LJ
// minimum, where g vanishes, b r^2 stays below ~1e3), so with gmax the largest |g| of the force
// pass of the same bead the bound is 8 max|eta| (16 gmax + 1e3).  The scale takes that bound
// below 2^24: shares stay inside the grid's range, which resolves them to 2^-42 of the largest.
__device__ __forceinline__ float bl_jscale(float etamax, float gmax) {
  if (!(etamax > 0.f)) return 1.f;
  const float bound = 8.f * etamax * fmaf(16.f, gmax, 1e3f);
  int e;
  const float f = frexpf(bound, &e);   // bound = f 2^e, f in [0.5, 1): bound < 2^e
  (void)f;
  return ldexpf(1.f, 24 - max(-90, min(120, e)));
}

// bit 8 jj of the result is set iff byte jj of m is nonzero
__device__ __forceinline__ unsigned long long nonzero_bytes(unsigned long long m) {
  m |= m >> 4;
  m |= m >> 2;
  m |= m >> 1;
  return m & 0x0101010101010101ull;
}

// One j-atom of the walk: coordinates minus the entry's Delta, eta, charge and type.
struct BLJ {
  float2 x[3], e[3];
  float2 qj;
  int tj;
};

// One unit: i-atoms ih * kBLI .. ih * kBLI + kBLI - 1 of i-cluster ci for beads 64 g + lane and
// 64 g + 32 + lane of the pass.
template <int MODE, bool EW, bool HALF>
__device__ __forceinline__ void bl_unit(const SysConsts& sc, BLWarp<MODE>& S, const PathDev& P, int g, int ci,
                                        int ih, int lane) {
  const int a0 = ih * kBLI;   // first i-atom of the unit within the cluster
  constexpr int NR = BLRow<MODE>::value;
  const int n_pass = MODE == 0 ? P.n_force : P.n_hvp;
  const int b0 = g * kBLBeads + lane, b1 = b0 + 32;
  const size_t gstride = (size_t)P.Qpad * 3 * 32;
  // element (slot s, component c) of this lane at base[(s * 3 + c) * 32]
  const float2* __restrict__ xg = P.xb + g * gstride + lane;
  const float2* __restrict__ eg = MODE >= 1 ? P.etab + g * gstride + lane : nullptr;
  BLConst k;
  k.drf = dup2(sc.drff);
  k.nk2rf = dup2(-sc.k2rff);
  k.ewb = sc.ewb;
  k.ewb2 = sc.ewb2;
  k.ewc2 = sc.ewc2;
  k.tew2 = dup2(2.f * sc.ewb2);
  float2 eps2 = make_float2(0.f, 0.f);
  if constexpr (MODE == 2) {
    // eps = h / max_i |eta_i| per bead (the largest atomic displacement is h)
    const float m0 = __uint_as_float(P.etamax[min(b0, n_pass - 1)]);
    const float m1 = __uint_as_float(P.etamax[min(b1, n_pass - 1)]);
    eps2 = make_float2((float)(m0 > 0.f ? sc.fd_h / (double)m0 : sc.fd_h),
                       (float)(m1 > 0.f ? sc.fd_h / (double)m1 : sc.fd_h));
  }
  // half list: a j-atom's share fj goes to the sums as -fj jmul (FD: in the units of H eta)
  float2 jmul = make_float2(1.f, 1.f);
  if constexpr (HALF && MODE >= 1) {
    const int c0 = min(b0, n_pass - 1), c1 = min(b1, n_pass - 1);
    jmul = make_float2(bl_jscale(__uint_as_float(P.etamax[c0]), __uint_as_float(P.gmax[c0])),
                       bl_jscale(__uint_as_float(P.etamax[c1]), __uint_as_float(P.gmax[c1])));
    if constexpr (MODE == 2) jmul = mul2(jmul, make_float2(-0.5f / eps2.x, -0.5f / eps2.y));
  }
  const float2 njmul = make_float2(-jmul.x, -jmul.y);
  float2 jbig = make_float2(0.f, 0.f);   // check build: the largest |share| of each bead
  float2 gm = make_float2(0.f, 0.f);   // force pass: largest |g| of each bead (scale of the H eta j-side sums)
  float2 xi[kBLI][3], ei[kBLI][3], acc[kBLI][3];
#pragma unroll
  for (int a = 0; a < kBLI; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = ((size_t)(ci * kCL + a0 + a) * 3 + c) * 32;
      xi[a][c] = __ldg(xg + o);
      if constexpr (MOP_BL_EISH && MODE >= 1) {
        S.ei[a * 3 + c][lane] = __ldg(eg + o);
        ei[a][c] = make_float2(0.f, 0.f);
      } else {
        ei[a][c] = MODE >= 1 ? __ldg(eg + o) : make_float2(0.f, 0.f);
      }
      acc[a][c] = make_float2(0.f, 0.f);
    }
  __syncwarp();
  for (int k2 = lane; k2 < kBLI * sc.n_types; k2 += 32) {
    const int i = k2 / sc.n_types, tj = k2 - i * sc.n_types;
    const int s = ci * kCL + a0 + i;
    const float qi = __ldg(&P.xq[s]).w;   // sqrt(f) q, the same in every bead's row
    const float4 t = __ldg(&sc.tab[__ldg(&P.ts[s]) * sc.n_types + tj]);
    float4* r = S.pt + (i * kMaxTypes + tj) * NR;
    r[0] = make_float4(t.x, t.x, -t.y, -t.y);
    r[1] = make_float4(qi, qi, t.z, t.z);
    if (NR == 3) r[2] = make_float4(14.f * t.x, 14.f * t.x, -8.f * t.y, -8.f * t.y);
  }
#pragma unroll
  for (int k2 = 0; k2 < 2 * kBLI * 3; ++k2) S.hl[k2][lane] = make_float2(0.f, 0.f);
  const int cnt = __ldg(&P.lcnt[ci]);
  const size_t eb = (size_t)ci * P.cap;
  int since_fold = 0;
  // qv, tv: lane jj < 8 holds the charge and pair-table offset of j-atom jj of the entry
  auto load_j = [&](int cj, int jj, BLJ& J, float qv, int tv) __attribute__((always_inline)) {
    const int sj = cj * kCL + jj;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = ((size_t)sj * 3 + c) * 32;
      if constexpr (MOP_BL_JCG) {
        J.x[c] = __ldcg(xg + o);
        if (MODE >= 1) J.e[c] = __ldcg(eg + o);
      } else {
        J.x[c] = __ldg(xg + o);
        if (MODE >= 1) J.e[c] = __ldg(eg + o);
      }
    }
    if constexpr (BLQtShfl<MODE>::value) {
      J.qj = dup2(__shfl_sync(0xffffffffu, qv, jj));
      J.tj = __shfl_sync(0xffffffffu, tv, jj);
    } else {
      (void)qv;
      (void)tv;
      J.qj = dup2(__ldg(&P.xq[sj]).w);
      J.tj = __ldg(&P.ts[sj]) * NR;
    }
  };
  auto prefetch_j = [&](int cj, int jj) __attribute__((always_inline)) {
    const int sj = cj * kCL + jj;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = ((size_t)sj * 3 + c) * 32;
      asm volatile("prefetch.global.L1 [%0];" ::"l"(xg + o));
      if (MODE >= 1) asm volatile("prefetch.global.L1 [%0];" ::"l"(eg + o));
    }
  };
  for (int c0 = 0; c0 < cnt; c0 += 32) {
    const int nc = min(32, cnt - c0);
    __syncwarp();
    if (lane < nc) {
      S.ent[lane] = __ldg(&P.ent[eb + c0 + lane]);
      S.m[lane] = __ldg(&P.emask[eb + c0 + lane]);
    }
    __syncwarp();
    for (int e = 0; e < nc; ++e) {
      const int4 E = S.ent[e];
      unsigned long long M = S.m[e];
      const int cj = E.x & kCluMask;
      if constexpr (HALF) {
        // each unordered cluster pair once: its owner entry, and a self entry's pairs j > i
        if (!(E.x & kOwnerFlag)) continue;   // warp-uniform
        if (E.x & kSelfFlag) M &= 0x7f3f1f0f07030100ull;
      }
      const float2 D[3] = {dup2(__int_as_float(E.y)), dup2(__int_as_float(E.z)), dup2(__int_as_float(E.w))};
      // this unit's candidate bits: i-atoms a0 .. a0 + kBLI - 1 of every j byte
      const unsigned long long Mi = (M >> a0) & (0x0101010101010101ull * ((1u << kBLI) - 1u));
      if (!Mi) continue;   // warp-uniform: no candidate pair for these i-atoms
      if constexpr (BLEpf<MODE>::value) {
        // the next entry of this chunk that the walk evaluates (warp-uniform scan in shared memory)
        unsigned long long Mn = 0ull;
        int cn = 0;
        for (int e2 = e + 1; e2 < nc && !Mn; ++e2) {
          const int x2 = S.ent[e2].x;
          unsigned long long M2 = S.m[e2];
          if (HALF) {
            if (!(x2 & kOwnerFlag)) continue;
            if (x2 & kSelfFlag) M2 &= 0x7f3f1f0f07030100ull;
          }
          Mn = (M2 >> a0) & (0x0101010101010101ull * ((1u << kBLI) - 1u));
          cn = x2 & kCluMask;
        }
        if (Mn) {
          // lane t < 24: line t % 6 of j-atom t / 6 (first instruction) or t / 6 + 4 (second)
          const int pj = lane / 6, pl = lane - 6 * pj;
          const char* bx = reinterpret_cast<const char*>(P.xb + g * gstride) + (size_t)cn * (kCL * 3 * 32 * 8) +
                           pj * (3 * 32 * 8) + pl * 128;
          const char* be = MODE >= 1 ? reinterpret_cast<const char*>(P.etab + g * gstride) +
                                           (size_t)cn * (kCL * 3 * 32 * 8) + pj * (3 * 32 * 8) + pl * 128
                                     : nullptr;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (lane < 24 && ((Mn >> (8 * (pj + 4 * h))) & 0xffull)) {
              asm volatile("prefetch.global.L1 [%0];" ::"l"(bx + h * (4 * 3 * 32 * 8)));
              if (MODE >= 1) asm volatile("prefetch.global.L1 [%0];" ::"l"(be + h * (4 * 3 * 32 * 8)));
            }
          }
        }
      }
      unsigned long long nz = nonzero_bytes(Mi);
      // charges and pair-table offsets of the entry's 8 j-atoms, one load per entry (the j-loop
      // takes them by shuffle instead of two dependent loads per j-atom)
      float qv = 0.f;
      int tv = 0;
      if (BLQtShfl<MODE>::value && lane < kCL) {
        qv = __ldg(&P.xq[cj * kCL + lane]).w;
        tv = __ldg(&P.ts[cj * kCL + lane]) * NR;
      }
      // evaluate the candidate pairs of one j-atom (the i-loop is unrolled: registers stay static)
      auto eval_j = [&](const BLJ& cur, int jj) __attribute__((always_inline)) {
        const unsigned byte = (unsigned)(Mi >> (8 * jj)) & 0xffu;
        float2 fj[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        float2 xj[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) xj[c] = sub2(cur.x[c], D[c]);
        const float4* pj = S.pt + cur.tj;   // row of i-atom i at pj[i * kMaxTypes * NR]
        auto pair = [&](int i) __attribute__((always_inline)) {
          const float4* tp = pj + i * kMaxTypes * NR;
          const float4 t0 = tp[0], t1 = tp[1];
          BLPair c;
          c.A = make_float2(t0.x, t0.y);
          c.nB = make_float2(t0.z, t0.w);
          c.qq = mul2(make_float2(t1.x, t1.y), cur.qj);
          c.sh = fma2(c.qq, k.drf, make_float2(t1.z, t1.w));
          if constexpr (MODE == 0) {
            bl_force<EW, HALF>(k, c, sc.rc2f, xi[i], xj, acc[i], fj, gm);
          } else {
            float2 eii[3];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) eii[cc] = MOP_BL_EISH ? S.ei[i * 3 + cc][lane] : ei[i][cc];
            if constexpr (MODE == 1) bl_hvp<EW, HALF>(k, c, sc.rc2f, tp[2], xi[i], xj, eii, cur.e, acc[i], fj);
            else bl_fd<EW, HALF>(k, c, sc.rc2f, eps2, xi[i], xj, eii, cur.e, acc[i], fj);
          }
        };
        // groups of kBLIlp i-atoms whose candidate bits are all set are evaluated together (their
        // dependency chains interleave); other groups one candidate at a time
#pragma unroll
        for (int i0 = 0; i0 < kBLI; i0 += kBLIlp) {
          constexpr unsigned gm = (1u << kBLIlp) - 1u;
          const unsigned bits = (byte >> i0) & gm;
          if (kBLIlp > 1 && bits == gm) {   // warp-uniform
#pragma unroll
            for (int i = i0; i < i0 + kBLIlp; ++i) pair(i);
          } else if (bits) {
#pragma unroll
            for (int i = i0; i < i0 + kBLIlp; ++i)
              if ((bits >> (i - i0)) & 1u) pair(i);   // warp-uniform
          }
        }
        if constexpr (HALF) {
          // the j-atom's share of these pairs, for both beads of the lane, with the sign reversed,
          // on the two grids of the exact j-side sums
          // [component][bead half][lane] words of the j-atom: 256 contiguous bytes per atomic
          unsigned long long* jp = P.jI + (g * (size_t)P.Qpad + (size_t)(cj * kCL + jj)) * 3 * 64 + lane;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            unsigned long long w0, w1;
            const float2 v = mul2(fj[q], njmul);
            if constexpr (MOP_BL_JCHECK)
              jbig = make_float2(fmaxf(jbig.x, fabsf(v.x)), fmaxf(jbig.y, fabsf(v.y)));
            bl_fix<MODE == 0 ? 0 : 1>(v, w0, w1);
            atomicAdd(jp + q * 64, w0);
            atomicAdd(jp + q * 64 + 32, w1);
          }
        }
      };
#if MOP_BL_JSTATIC
      // j-atoms in a fixed, unrolled order: offsets are constants, no bookkeeping
      (void)nz;
      if constexpr ((MODE == 0 && MOP_BL_JPF_F) || (MODE != 0 && MOP_BL_JPF_H)) {
      // software pipeline: the next j-atom's loads are issued before the current one is
      // evaluated (after unrolling, handing the registers on costs nothing)
      BLJ cur;
      if ((Mi & 0xffull) != 0ull) load_j(cj, 0, cur, qv, tv);
#pragma unroll
      for (int jj = 0; jj < kCL; ++jj) {
        BLJ nxt;
        if (jj + 1 < kCL && ((Mi >> (8 * (jj + 1))) & 0xffull)) load_j(cj, jj + 1, nxt, qv, tv);   // warp-uniform
        if ((Mi >> (8 * jj)) & 0xffull) eval_j(cur, jj);
        cur = nxt;
      }
      } else {
#pragma unroll (BLJUnroll<MODE, HALF>::value)
      for (int jj = 0; jj < kCL; ++jj) {
        if (!((Mi >> (8 * jj)) & 0xffull)) continue;   // warp-uniform
        if constexpr (MOP_BL_L1PF) {
          // the next j-atom's rows move towards L1 while this one is evaluated (no registers)
          if (jj + 1 < kCL && ((Mi >> (8 * (jj + 1))) & 0xffull)) prefetch_j(cj, jj + 1);
        }
        BLJ cur;
        load_j(cj, jj, cur, qv, tv);
        eval_j(cur, jj);
      }
      }
#else
      int jj = (__ffsll((long long)nz) - 1) >> 3;
      nz &= nz - 1;
      BLJ cur;
      load_j(cj, jj, cur, qv, tv);
      while (true) {
        // the next j-atom of this entry is loaded while the current one is evaluated
        const bool more = nz != 0ull;
        BLJ nxt;
        int jn = 0;
        if (more) {
          jn = (__ffsll((long long)nz) - 1) >> 3;
          nz &= nz - 1;
          load_j(cj, jn, nxt, qv, tv);
        }
        eval_j(cur, jj);
        if (!more) break;
        cur = nxt;
        jj = jn;
      }
#endif
      if (++since_fold == kBLFold) {
        bl_fold(S, acc, lane);
        since_fold = 0;
      }
    }
  }
  bl_fold(S, acc, lane);
  const bool v0 = b0 < n_pass, v1 = b1 < n_pass;
  // check build: poison the rows of a bead whose shares left the promised range
  const float jlim = MODE == 0 ? 1073741824.f : 16777216.f;
  const bool bad0 = MOP_BL_JCHECK && !(jbig.x <= jlim), bad1 = MOP_BL_JCHECK && !(jbig.y <= jlim);
  if constexpr (MODE == 0) {
    // non-negative floats order like their bit patterns
    if (v0) atomicMax(&P.gmax[b0], __float_as_uint(gm.x));
    if (v1) atomicMax(&P.gmax[b1], __float_as_uint(gm.y));
  }
#pragma unroll
  for (int a = 0; a < kBLI; ++a) {
    const int s = ci * kCL + a0 + a;
    float2 h[3], l[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h[c] = S.hl[a * 3 + c][lane];
      l[c] = S.hl[3 * kBLI + a * 3 + c][lane];
    }
    if constexpr (MODE == 0) {
      float2* F = reinterpret_cast<float2*>(P.Fnb);
      if (v0) {
        float2* dst = F + 3 * ((size_t)b0 * P.Qpad + s);
#pragma unroll
        for (int c = 0; c < 3; ++c) dst[c] = bad0 ? make_float2(__int_as_float(0x7fc00000), 0.f) : make_float2(h[c].x, l[c].x);
      }
      if (v1) {
        float2* dst = F + 3 * ((size_t)b1 * P.Qpad + s);
#pragma unroll
        for (int c = 0; c < 3; ++c) dst[c] = bad1 ? make_float2(__int_as_float(0x7fc00000), 0.f) : make_float2(h[c].y, l[c].y);
      }
    } else {
      // H eta of the pair terms in FP32; FD: -(F(+) - F(-)) / (2 eps)
      const float2 sc2 = MODE == 2 ? make_float2(-0.5f / eps2.x, -0.5f / eps2.y) : make_float2(1.f, 1.f);
      float4* H = reinterpret_cast<float4*>(P.Hnb);
      const float poison = __int_as_float(0x7fc00000);
      if (v0)
        H[(size_t)b0 * P.Qpad + s] = bad0 ? make_float4(poison, poison, poison, 0.f)
                                          : make_float4((h[0].x + l[0].x) * sc2.x, (h[1].x + l[1].x) * sc2.x,
                                                        (h[2].x + l[2].x) * sc2.x, 0.f);
      if (v1)
        H[(size_t)b1 * P.Qpad + s] = bad1 ? make_float4(poison, poison, poison, 0.f)
                                          : make_float4((h[0].y + l[0].y) * sc2.y, (h[1].y + l[1].y) * sc2.y,
                                                        (h[2].y + l[2].y) * sc2.y, 0.f);
    }
  }
}

// resident blocks per SM asked of the register allocator: 20 warps (96 registers) for the
// force kernel, 16 (128 registers) for the HVP kernel, and for the FD kernel (two force
// evaluations per pair) MOP_BL_MINB_D
#ifndef MOP_BL_MINB_F
#define MOP_BL_MINB_F (20 / MOP_BL_WARPS_F)
#endif
#ifndef MOP_BL_MINB_H
#define MOP_BL_MINB_H (16 / MOP_BL_WARPS_H)
#endif
#ifndef MOP_BL_MINB_D
#define MOP_BL_MINB_D (12 / MOP_BL_WARPS_H)
#endif
// half list: 16 warps (128 registers) for the force and HVP kernels, 12 for the FD kernel
#ifndef MOP_BL_MINB_FH
#define MOP_BL_MINB_FH (16 / MOP_BL_WARPS_F)
#endif
#ifndef MOP_BL_MINB_HH
#define MOP_BL_MINB_HH (16 / MOP_BL_WARPS_H)
#endif
#ifndef MOP_BL_MINB_DH
#define MOP_BL_MINB_DH (12 / MOP_BL_WARPS_H)
#endif
template <int MODE, bool HALF> struct BLMinBlocks {
  static constexpr int value = HALF ? (MODE == 0 ? MOP_BL_MINB_FH : (MODE == 1 ? MOP_BL_MINB_HH : MOP_BL_MINB_DH))
                                    : (MODE == 0 ? MOP_BL_MINB_F : (MODE == 1 ? MOP_BL_MINB_H : MOP_BL_MINB_D));
};

template <bool EW>
__device__ __forceinline__ void energy1_warp(const SysConsts& sc, const PathDev& P, int ci, int lane, int4* sent,
                                             unsigned long long* sm);

// e1_clu > 0 (force pass over the full list): units n_units .. n_units + n_paths e1_clu - 1 are the
// bead-1 pair energy of cluster (u - n_units) % e1_clu of path (u - n_units) / e1_clu
template <int MODE, bool EW, bool HALF>
__global__ void __launch_bounds__(32 * BLWarps<MODE>::value, BLMinBlocks<MODE, HALF>::value)
    k_pairb(SysConsts sc, const PathDev* __restrict__ paths, int n_paths, long long n_units, int e1_clu) {
  extern __shared__ __align__(16) unsigned char smem[];
  BLWarp<MODE>* W = reinterpret_cast<BLWarp<MODE>*>(smem);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long u = (long long)blockIdx.x * BLWarps<MODE>::value + w;
  if constexpr (MODE == 0 && !HALF) {
    if (u >= n_units && e1_clu > 0) {
      const long long e = u - n_units;
      const int p = (int)(e / e1_clu), ci = (int)(e - (long long)p * e1_clu);
      if (p >= n_paths) return;
      const PathDev& P = paths[p];
      if (ci >= __ldg(&P.meta[0])) return;   // warp-uniform
      energy1_warp<EW>(sc, P, ci, lane, W[w].ent, W[w].m);
      return;
    }
  }
  if (u >= n_units) return;
  int p = 0;
  if (MODE == 0) {
    while (p + 1 < n_paths && paths[p + 1].unit_off <= u) ++p;
  } else {
    while (p + 1 < n_paths && paths[p + 1].unit_off_h <= u) ++p;
  }
  const PathDev& P = paths[p];
  // group-major: the warps of a block take consecutive units (cluster halves, clusters) of the
  // same bead group
  const long long v = u - (MODE == 0 ? P.unit_off : P.unit_off_h);
  const long long per_group = (long long)P.n_clu * kBLSplit;
  const int g = (int)(v / per_group);
  const int r = (int)(v - g * per_group), ci = r / kBLSplit, ih = r - ci * kBLSplit;
  if (ci >= __ldg(&P.meta[0])) return;   // past the clusters of the current sort
  bl_unit<MODE, EW, HALF>(sc, W[w], P, g, ci, ih, lane);
}

template <int MODE, bool EW, bool HALF>
cudaError_t launch_b(const SysConsts& sc, const PathDev* d_paths, int n_paths, long long n_units, Launch L,
                     int e1_clu = 0) {
  constexpr int W = BLWarps<MODE>::value;
  const size_t smem = sizeof(BLWarp<MODE>) * W;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_pairb<MODE, EW, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long n_e1 = (MODE == 0 && !HALF && e1_clu > 0) ? (long long)n_paths * e1_clu : 0;
  const long long blocks = (n_units + n_e1 + W - 1) / W;
  k_pairb<MODE, EW, HALF><<<(unsigned)blocks, 32 * W, smem, L.st>>>(sc, d_paths, n_paths, n_units,
                                                                     n_e1 > 0 ? e1_clu : 0);
  ++*L.counter;
  return cudaGetLastError();
}

// ---- bead-1 pair energy --------------------------------------------------------------------
// One warp per i-cluster, lane (i = lane & 7, jq = lane >> 3) against j-atoms jq and jq + 4 of
// every owner entry (a self entry's pairs j > i), so each pair is met once.
// phi_sf(r) = phi(r) - phi(rc) - (r - rc) phi'(rc) (sh = phi'(rc) = 0 with the potential shift).
// One warp: i-cluster ci of path P; sent and sm hold the warp's chunk of 32 list entries.
template <bool EW>
__device__ __forceinline__ void energy1_warp(const SysConsts& sc, const PathDev& P, int ci, int lane, int4* sent,
                                             unsigned long long* sm) {
  const int i = lane & 7, jq = lane >> 3;
  const int si = ci * kCL + i;
  const float4 xi = __ldg(&P.xq[si]);   // bead 1 is row 0
  const int ti = __ldg(&P.ts[si]);
  const int cnt = __ldg(&P.lcnt[ci]);
  const size_t eb = (size_t)ci * P.cap;
  float acc = 0.f, hi = 0.f, lo = 0.f;
  for (int c0 = 0; c0 < cnt; c0 += 32) {
    // the warp loads 32 entries at once; the j-atom loads of an entry then depend on a
    // shared-memory read only
    const int nc = min(32, cnt - c0);
    __syncwarp();
    if (lane < nc) {
      sent[lane] = __ldg(&P.ent[eb + c0 + lane]);
      sm[lane] = __ldg(&P.emask[eb + c0 + lane]);
    }
    __syncwarp();
    for (int e = 0; e < nc; ++e) {
      const int4 E = sent[e];
      if (!(E.x & kOwnerFlag)) continue;   // warp-uniform
      unsigned long long M = sm[e];
      if (E.x & kSelfFlag) M &= 0x7f3f1f0f07030100ull;
      const int cj = E.x & kCluMask;
      const float Dx = __int_as_float(E.y), Dy = __int_as_float(E.z), Dz = __int_as_float(E.w);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = jq + 4 * h;
        if (!((M >> (j * kCL + i)) & 1ull)) continue;
        const int sj = cj * kCL + j;
        const float4 xj = __ldg(&P.xq[sj]);
        const float4 p = __ldg(&sc.tab[ti * sc.n_types + __ldg(&P.ts[sj])]);
        const float dx = xi.x + Dx - xj.x, dy = xi.y + Dy - xj.y, dz = xi.z + Dz - xj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(r2 < sc.rc2f)) continue;
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float rinv6 = rinv * rinv * rinv * rinv * rinv * rinv;
        const float qq = xi.w * xj.w;
        const float sh = fmaf(qq, sc.drff, p.z);
        const float elj = rinv6 * fmaf(p.x * (1.f / 12.f), rinv6, -p.y * (1.f / 6.f));
        float el;
        if constexpr (EW) {
          const float x = sc.ewb * r;
          const float ec = ex2_approx(-sc.ewb2 * r2 * 1.4426950408889634f) * erfcx_rational(x);
          el = qq * fmaf(ec, rinv, -sc.ewec);
        } else {
          el = qq * (rinv + fmaf(sc.krff, r2, -sc.crff));
        }
        acc += elj + el - p.w - (r - sc.rcf) * sh;
      }
    }
    two_sum_add(hi, lo, acc);
    acc = 0.f;
  }
  two_sum_add(hi, lo, acc);
  const df v = df_warp_sum(df{hi, lo});
  if (lane == 0) P.e_pair[ci] = (double)v.hi + (double)v.lo;
}

template <bool EW>
__global__ void __launch_bounds__(128) k_energy1(SysConsts sc, const PathDev* __restrict__ paths, int max_clu) {
  __shared__ int4 sent[4][32];
  __shared__ unsigned long long sm[4][32];
  const PathDev& P = paths[blockIdx.y];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ci = blockIdx.x * 4 + w;
  if (ci >= max_clu || ci >= __ldg(&P.meta[0])) return;   // warp-uniform
  energy1_warp<EW>(sc, P, ci, lane, sent[w], sm[w]);
}

// ---- transposition into the bead-lane layout -------------------------------------------------
// Block (cluster c, group g): 64 bead rows x 8 slots of src through shared memory into the
// 8 x 3 x 32 float2 of dst, which are contiguous.
__global__ void __launch_bounds__(256) k_bl_transpose(const float4* __restrict__ src, int n_valid, int Qpad,
                                                      int max_clu, const int* meta, float2* __restrict__ dst) {
  __shared__ float4 t[kBLBeads][kCL];
  const int c = blockIdx.x, g = blockIdx.y;
  if (c >= max_clu || c >= __ldg(&meta[0])) return;   // block-uniform
  for (int k = threadIdx.x; k < kBLBeads * kCL; k += blockDim.x) {
    const int b = k / kCL, a = k - b * kCL;
    const int row = min(g * kBLBeads + b, n_valid - 1);
    t[b][a] = __ldg(&src[(size_t)row * Qpad + c * kCL + a]);
  }
  __syncthreads();
  float2* out = dst + ((size_t)g * Qpad + (size_t)c * kCL) * 3 * 32;
  for (int k = threadIdx.x; k < kCL * 3 * 32; k += blockDim.x) {
    const int l = k & 31, ac = k >> 5, a = ac / 3, comp = ac - 3 * a;
    const float4 p = t[l][a], q = t[l + 32][a];
    out[k] = comp == 0 ? make_float2(p.x, q.x) : (comp == 1 ? make_float2(p.y, q.y) : make_float2(p.z, q.z));
  }
}

// ---- j-side sums of the half list into the rows -----------------------------------------------
// Block (cluster c, group g, path): the 8 slots x 64 beads of jF through shared memory; force
// rows are double-floats (TwoSum of the high part with the FP32 sum), H eta rows FP32.
// The fixed-point sums are added to the rows: to the double-float forces exactly rounded, to the
// FP32 H eta rows divided by the bead's scale (a power of two).
template <int MODE>
__global__ void __launch_bounds__(256) k_bl_combine(SysConsts sc, const PathDev* __restrict__ paths) {
  (void)sc;
  __shared__ unsigned long long t[kCL * 3][64];
  const PathDev& P = paths[blockIdx.z];
  const int c = blockIdx.x, g = blockIdx.y;
  const int rows = MODE == 0 ? P.n_force : P.n_hvp;
  if (c >= P.n_clu || c >= __ldg(&P.meta[0]) || g * kBLBeads >= rows) return;   // block-uniform
  const size_t o = ((size_t)g * P.Qpad + (size_t)c * kCL) * 3 * 64;
  for (int k = threadIdx.x; k < kCL * 3 * 64; k += blockDim.x) t[k >> 6][k & 63] = P.jI[o + k];
  __syncthreads();
  for (int k = threadIdx.x; k < kBLBeads * kCL; k += blockDim.x) {
    const int bb = k / kCL, a = k - bb * kCL;
    const int b = g * kBLBeads + bb;
    if (b >= rows) continue;
    // bead bb is half bb / 32 of lane bb % 32
    const int l = (bb & 31) + (bb & 32);
    const size_t s = (size_t)c * kCL + a;
    if constexpr (MODE == 0) {
      // forces: (hi + lo + j) rounded to a double-float, in FP64 (hi + lo is exact there)
      float2* F = reinterpret_cast<float2*>(P.Fnb) + 3 * ((size_t)b * P.Qpad + s);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float2 f = F[q];
        const double sum = ((double)f.x + (double)f.y) + bl_unfix<0>(t[a * 3 + q][l]);
        const float nh = (float)sum;
        F[q] = make_float2(nh, (float)(sum - (double)nh));
      }
    } else {
      // H eta rows are FP32: the sums are decoded in FP32 (the FP64 pipe of this part would make
      // the decode the bound of the pass), divided by the bead's scale (a power of two)
      const float inv = 1.f / bl_jscale(__uint_as_float(P.etamax[b]), __uint_as_float(P.gmax[b]));
      float j[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const unsigned long long w = t[a * 3 + q][l];
        const int lo = (int)(unsigned)(w & 0xffffffffull);
        const int hi = (int)(((long long)w - (long long)lo) >> 32);
        j[q] = fmaf(__int2float_rn(hi), BLGrid<1>::kHi, __int2float_rn(lo) * (1.f / BLGrid<1>::kLo)) * inv;
      }
      float4* H = reinterpret_cast<float4*>(P.Hnb) + (size_t)b * P.Qpad + s;
      float4 h = *H;
      h.x += j[0];
      h.y += j[1];
      h.z += j[2];
      *H = h;
    }
  }
}

}  // namespace

int pairb_units_per_cluster() { return kBLSplit; }

cudaError_t launch_bl_combine(const SysConsts& sc, const PathDev* d_paths, const PathDev* h_paths, int n_paths,
                              int mode, Launch L) {
  int groups = 0, clu = 0;
  for (int p = 0; p < n_paths; ++p) {
    groups = std::max(groups, bl_groups(mode == 0 ? h_paths[p].n_force : h_paths[p].n_hvp));
    clu = std::max(clu, h_paths[p].n_clu);
  }
  if (groups == 0 || clu == 0) return cudaSuccess;
  const dim3 grid((unsigned)clu, (unsigned)groups, (unsigned)n_paths);
  if (mode == 0) k_bl_combine<0><<<grid, 256, 0, L.st>>>(sc, d_paths);
  else if (mode == 1) k_bl_combine<1><<<grid, 256, 0, L.st>>>(sc, d_paths);
  else k_bl_combine<2><<<grid, 256, 0, L.st>>>(sc, d_paths);
  ++*L.counter;
  return cudaGetLastError();
}

bool pairb_fuses_energy1(const SysConsts& sc) { return MOP_BL_E1FUSE && (sc.bl == 1 || sc.bl == 3); }

cudaError_t launch_pairb(const SysConsts& sc, const PathDev* d_paths, int n_paths, long long n_units, int mode,
                         Launch L, int e1_clu) {
  if (n_units <= 0) return cudaSuccess;
  const bool ew = sc.elec == 1;
  // j-side sums: the half list in both passes, the owner entries of the full list in the H eta pass
  const bool half = mode == 0 ? sc.bl == 2 : (sc.bl == 1 || sc.bl == 2);
  if (half) {
    switch (mode) {
      case 0: return ew ? launch_b<0, true, true>(sc, d_paths, n_paths, n_units, L) : launch_b<0, false, true>(sc, d_paths, n_paths, n_units, L);
      case 1: return ew ? launch_b<1, true, true>(sc, d_paths, n_paths, n_units, L) : launch_b<1, false, true>(sc, d_paths, n_paths, n_units, L);
      default: return ew ? launch_b<2, true, true>(sc, d_paths, n_paths, n_units, L) : launch_b<2, false, true>(sc, d_paths, n_paths, n_units, L);
    }
  }
  switch (mode) {
    case 0: return ew ? launch_b<0, true, false>(sc, d_paths, n_paths, n_units, L, e1_clu)
                      : launch_b<0, false, false>(sc, d_paths, n_paths, n_units, L, e1_clu);
    case 1: return ew ? launch_b<1, true, false>(sc, d_paths, n_paths, n_units, L) : launch_b<1, false, false>(sc, d_paths, n_paths, n_units, L);
    default: return ew ? launch_b<2, true, false>(sc, d_paths, n_paths, n_units, L) : launch_b<2, false, false>(sc, d_paths, n_paths, n_units, L);
  }
}

cudaError_t launch_energy1(const SysConsts& sc, const PathDev* d_paths, int n_paths, int max_clu, Launch L) {
  const dim3 grid((unsigned)((max_clu + 3) / 4), (unsigned)n_paths);
  if (sc.elec == 1) k_energy1<true><<<grid, 128, 0, L.st>>>(sc, d_paths, max_clu);
  else k_energy1<false><<<grid, 128, 0, L.st>>>(sc, d_paths, max_clu);
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_bl_transpose(const float4* src, int n_valid, int Qpad, int max_clu, const int* meta, float2* dst,
                                Launch L) {
  if (n_valid <= 0) return cudaSuccess;
  const dim3 grid((unsigned)max_clu, (unsigned)bl_groups(n_valid));
  k_bl_transpose<<<grid, 256, 0, L.st>>>(src, n_valid, Qpad, max_clu, meta, dst);
  ++*L.counter;
  return cudaGetLastError();
}

}  // namespace mop
