// Internal declarations shared by the CUDA translation units of libmop.
//
// Data layout in HBM (per path p with N beads, Q atoms, Qpad = 8 * n_clu slots):
//   x32/x64 [N][Q][3]      caller-order coordinates (the path state)
//   perm[Qpad], slot[Q]    spatial order: slot -> atom (-1 = padding), atom -> slot
//   xq/xq64 [N][Qpad]      cluster-local coordinates (x - C_cluster) and sqrt(f) q
//   ent/ent64/emask [E]    cluster-pair list shared by all beads of the path
//   Fnb, F, eta, Hnb, Heta [N][Qpad][3] FP64 fields in slot order; eta32 [N][Qpad] float4
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mop {

constexpr int kCL = 8;            // atoms per cluster
constexpr int kMaxTypes = 16;
constexpr int kMaxPaths = 64;
constexpr int kMaxGroup = 1024;   // atoms per CV group
constexpr int kMaxGauss = 4096;   // Gaussians per path
constexpr int kMaxCV = 4;         // collective variables per path (multivariate Gaussians)
constexpr int kRedBlock = 256;    // threads of the elementwise kernels
constexpr double kCoulombF = 138.935458;   // kJ mol^-1 nm e^-2
constexpr double kBoltz = 0.0083144626;    // kJ mol^-1 K^-1
constexpr float kDummyCoord = 1.0e5f;      // padding slots sit far outside every cutoff
// list entry word x: j-cluster index | self-entry flag << 28 | half mask << 29 | exclusions << 31
constexpr int kCluMask = 0x0fffffff;
constexpr int kSelfFlag = 1 << 28;
// bead-lane lists: the entry that owns its unordered cluster pair (of an entry and its mirror
// image in the full list, one; every entry of the half list)
constexpr int kOwnerFlag = (int)0x80000000;
// j-side sums of the half-list pair kernels are fixed point with 23 fractional bits in int64:
// integer addition makes the atomics order-independent, so results stay bitwise reproducible
constexpr float kFixScale = 8388608.0f;           // 2^23
constexpr float kFixInv = 1.0f / 8388608.0f;
// Bead-lane pair kernels (mixed precision): one warp evaluates one i-cluster for a group of 64
// beads, lane l holding beads 64 g + l and 64 g + 32 + l as the two halves of f32x2 operands.
// Their coordinates and eta are kept transposed, float2 [group][slot][3][32], so that a warp
// reads one component of one atom for all 64 beads as 256 contiguous bytes.
constexpr int kBLBeads = 64;

// System-wide constants, passed by value to kernels.
struct SysConsts {
  int Q, n_types, cutoff_mode, precision, hvp_mode;
  double L[3], invL[3];
  float Lf[3], halfLf[3];
  float invLf[3];
  float Llo[3];   // L - Lf: the box as a double-float (Lf, Llo)
  double rc, rc2, krf, crf, k2rf, drf;   // RF constants; drf = phi'_RF(rc) / (f qi qj) if shifted
  float rcf, rc2f, krff, crff, k2rff, drff;
  double fd_h;
  // Ewald electrostatics (elec = 1): erfc(beta r)/r in the pair kernels, the erf correction of
  // excluded pairs, the self term, and the SPME reciprocal part
  int elec;
  float ewb, ewb2, ewc2, ewec;   // beta, beta^2, 2 beta / sqrt(pi), erfc(beta rc) / rc
  double e_self;                 // -f beta / sqrt(pi) sum_i q_i^2
  int n_excl;                    // excluded pairs (i < j, caller indices)
  const int* excl_off;           // atom a's excluded partners: excl_nb[excl_off[a] .. excl_off[a + 1])
  const int* excl_nb;
  // smooth particle-mesh Ewald (pme_nk == 0: no reciprocal part)
  int pme_order;
  int pme_K[3];
  int pme_kc3;                   // K3 / 2 + 1 (complex points along the last axis)
  long long pme_nk, pme_nkc;     // real and complex points of one grid
  float2 pme_kl[3];              // K / L as double-floats
  const float* pme_theta;        // [K1][K2][K3 / 2 + 1] Ewald kernel times the B-spline moduli
  // per-atom arrays in caller order
  const double* mass;
  const double* Kspr;   // m nu / (2 dt)
  const double* cL;     // dt / (m nu)
  const double* qs;     // q sqrt(f)
  const float2* c_df;   // c_i as a double-float (hi, lo) pair
  const float2* K_df;   // K_i as a double-float (hi, lo) pair
  const int* type;
  const int* mol;
  const int* loc;
  // bonded incidence: for atom a, terms inc[inc_off[a] .. inc_off[a+1])
  const int* inc_off;
  const int4* inc;      // x = kind (0 bond, 1 angle) | role << 2, y,z,w = atoms (w = -1 for bonds)
  const double2* incp;  // (r0 or theta0, k)
  const float2* incpf;  // the same in FP32 (mixed precision)
  // type-pair tables: (12 c12, 6 c6, phi'_LJ(rc) if shifted else 0, phi_LJ(rc))
  const float4* tab;
  const double4_32a* tab64;
  // mixed precision, bead-lane pair kernels on lists whose entries carry a 64-bit mask of the
  // candidate atom pairs (emask bit j * 8 + i: the atoms' union spheres come within rc and the
  // pair is not excluded).  1 = full list (every cluster pair from both sides); the force pass
  // evaluates every entry, the H eta pass only the owner entries, adding the j-atoms' shares to
  // exact fixed-point sums; 2 = half list for both passes; 3 = full list, every entry in both
  // passes (no j-side sums).  0 = the earlier half-list kernels.
  int bl;
};

// Device view of one path of a multi-path launch.
struct PathDev {
  // Qpad is the slot stride of every [bead][slot] array (8 x the cluster-count upper bound);
  // n_clu is that upper bound; the clusters of the current sort are meta[0] <= n_clu.
  int N, n_force, n_hvp, Q, Qpad, n_clu;
  const int* meta;
  long long unit_off;      // first force-kernel unit of this path
  long long unit_off_h;    // first HVP-kernel unit of this path
  int blk_off_e1, blk_off_e2;
  const float* x32;
  const double* x64;
  const int* perm;
  const int* slot;
  const float4* xq;
  const double4_32a* xq64;
  const int* ts;
  const int* lcnt;          // list length of each i-cluster
  int cap;                  // entries of cluster ci start at ci * cap
  const unsigned* ctype;    // packed LJ types of each cluster (4 bits per atom)
  const int4* ent;          // x = cj | self << 28 | half mask << 29 | has-exclusions << 31 (bead-lane
                            // lists: owner << 31); y,z,w = FP32 Delta
  const double4_32a* ent64;
  const unsigned long long* emask;   // excluded atom pairs of an entry (bit j * 8 + i), or with
                                     // bead-lane kernels the candidate pairs of the entry
  // bead-lane kernels: coordinates (cluster-local) and eta transposed, float2 [G][Qpad][3][32]
  // with G = ceil(beads / 64); element (g, s, c, l) = (bead 64 g + l, bead 64 g + 32 + l)
  const float2* xb;
  const float2* etab;
  // bead-lane j-side sums of the current pass: 64-bit fixed-point words [G][Qpad][3][2][32]
  // (component, bead half, lane; see mop_pairb.cu), zeroed before the pass
  unsigned long long* jI;
  // FP64 mode: [N][Qpad][3] doubles.  Mixed mode views of the same buffers: Fnb and F as
  // double-float (hi, lo) x 3 (float2 [N][Qpad][3]), Hnb and Heta as float4 [N][Qpad].
  double* Fnb;
  double* F;
  double* eta;
  float4* eta32;
  float4* etalo;           // mixed mode: eta - eta32 (eta as the double-float eta32 + etalo)
  double* Hnb;
  double* Heta;
  unsigned* etamax;        // [N] float bits of max_i |eta_i|
  unsigned* gmax;          // [N] float bits of the largest |g| of the force pass (bead-lane half list)
  // mixed mode: the list holds each cluster pair once and the pair kernels add the j-side sums
  // here, fixed point (kFixScale), [n_pass][Qpad][3]; NULL in FP64 mode (full list)
  unsigned long long* jacc;
  double* e_pair;          // [n_clu]
  double* grad;            // [N][Q][3] caller order
  // bias on n_cv CVs: CV d is the distance of the centres of groups gA[cv_a[d] .. cv_a[d + 1])
  // and gB[cv_b[d] .. cv_b[d + 1]) (end-to-end form of Eq. 8 with cv_e2e, mass-weighted with
  // cv_com); Gaussians k < n_gauss have centres gc[k][kMaxCV], widths gw[k][kMaxCV], height gh[k]
  int n_cv, n_gauss;
  int cv_a[kMaxCV + 1], cv_b[kMaxCV + 1];
  int cv_e2e[kMaxCV], cv_com[kMaxCV];
  double cv_width[kMaxCV];  // width of the Gaussians mop_metadynamics deposits (0: the call's)
  const int* gA;
  const int* gB;
  double* gc;
  double* gw;
  double* gh;
  double* e_excl;          // Ewald: bead-1 energy partials of the exclusion corrections
  const float2* cwdf;      // wrapped cluster centres as double-floats [n_clu][3]
  unsigned long long* pme_q;   // SPME: fixed-point charge grids [beads][nk]
  float2* pme_c;               // half spectra [beads][nkc]
  float* pme_phi;              // potential grids of the force pass [beads][nk]
  float* pme_phd;              // potential grids of the derivative grids (HVP pass) [beads][nk]
  double* pme_e;               // bead-1 energy partials
  double* diag;            // [8]: U1, E_spring, E_bias, CV, V_eff, U_pair, U_bonded
  double* veff_out;        // one double
};

// ------------------------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed tree); every thread must call it.  Result valid in thread 0.
template <int BS>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < BS / 32) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// Knuth's TwoSum: (hi, lo) += a without loss (FP32 error-free transformation).
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float a) {
  const float s = hi + a;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (a - bp);
  hi = s;
  lo += err;
}

// Double-float (hi + lo, |lo| <= ulp(hi)/2) helpers: FP64-class accuracy on the FP32 pipes.
// B300 issues FP64 at a small fraction of the FP32 rate, so the mixed-precision path keeps
// its extended-precision steps in this form (error-free transformations: Knuth's TwoSum,
// Dekker's FastTwoSum, and TwoProd through a fused multiply-add).
struct df {
  float hi, lo;
};
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return {s, (a - (s - bp)) + (b - bp)};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ df df_add_f(df x, float b) {
  df s = two_sum(x.hi, b);
  return fast_two_sum(s.hi, s.lo + x.lo);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ df df_from_double(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
// warp sum of a double-float value (fixed butterfly order)
__device__ __forceinline__ df df_warp_sum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, w);
  }
  return v;
}

// float -> double widening on the integer pipes (exact for normal numbers, zero, inf and NaN;
// FP32 subnormals are flushed to zero, as -ftz does).  B300 runs F2F conversions on its slow
// FP64 path, which made them the bottleneck of the elementwise kernels.
__device__ __forceinline__ double widen(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned sign = u & 0x80000000u, ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  unsigned hi, lo;
  if (ex == 0u) {
    hi = sign;
    lo = 0u;
  } else if (ex == 0xffu) {
    hi = sign | 0x7ff00000u | (man >> 3);
    lo = man << 29;
  } else {
    hi = sign | ((ex + 896u) << 20) | (man >> 3);
    lo = man << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double aligned_coord(double v, double ref, double L, double invL) {
  return v - L * rint((v - ref) * invL);
}

// fixed-point j-side sum (kFixScale units) as a double-float: hi is the value rounded to FP32,
// lo the exact integer remainder rounded to FP32
__device__ __forceinline__ df fix_to_df(long long v) {
  const float hi = __ll2float_rn(v);
  const long long r = v - __float2ll_rn(hi);
  return df{hi * kFixInv, __ll2float_rn(r) * kFixInv};
}

}  // namespace mop

