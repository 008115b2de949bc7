// Smooth particle-mesh Ewald (reciprocal space) for every bead of a path (MOP_ELEC_PME).
//
// Essmann et al., J. Chem. Phys. 103, 8577 (1995): charges are spread with cardinal B-splines of
// order P onto a K1 x K2 x K3 grid of the orthorhombic box, the grid is convolved with the Ewald
// reciprocal kernel theta(m) = exp(-pi^2 |m~|^2 / beta^2) / (pi V |m~|^2) |b(m)|^2 by a real
// FFT, and forces are gathered from the potential grid with the splines' derivatives.  The
// adjoint Hessian-vector product needs one more spread (of the charge grid's derivative along
// eta), one more FFT pair, and a gather with second derivatives of the splines:
//     (H eta)_i = q_i sum_k [(eta_i . grad) grad M_i](k) phi(k) + q_i sum_k grad M_i(k) phi'(k),
// with phi the potential grid of the force pass and phi' that of the derivative grid.
// Grids of charges are summed as int64 fixed point, so results do not depend on the order of
// the atomics; forces go into the path's fixed-point j-side sums.  The FFT convolution (grid ->
// spectrum -> times theta -> potential) is the batched transform of mop_fft.cu.
#include <algorithm>

#include "mop_host.h"

namespace mop {

// twiddle tables and radix plans of the three grid axes, made outside any stream capture
struct PmePlans {
  DevBuf<float2> tw[3];
  FftAxis ax[3];
  bool ready = false;
  ~PmePlans() {
    for (auto& t : tw) t.release();
  }
};

namespace {

constexpr float kGridFixF = 1099511627776.0f;       // 2^40: fixed-point unit of the grids
constexpr float kGridInv = 1.0f / 1099511627776.0f;

// B-spline values M_P(w + t), t = 0..P-1 (w in [0, 1)), and the first and second derivatives
// M_P' = M_{P-1}(x) - M_{P-1}(x - 1), M_P'' = M_{P-2}(x) - 2 M_{P-2}(x - 1) + M_{P-2}(x - 2), by
// the recursion M_n(x) = (x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)) / (n - 1).
template <int P>
__device__ __forceinline__ void spline(float w, float* M, float* dM, float* d2M) {
  float A[P + 1], Am1[P + 1], Am2[P + 1];
#pragma unroll
  for (int t = 0; t <= P; ++t) A[t] = Am1[t] = Am2[t] = 0.f;
  A[0] = w;
  A[1] = 1.f - w;
#pragma unroll
  for (int n = 2; n < P; ++n) {
#pragma unroll
    for (int t = 0; t <= P; ++t) {
      Am2[t] = Am1[t];
      Am1[t] = A[t];
    }
    float B[P + 1];
#pragma unroll
    for (int t = 0; t <= P; ++t) {
      const float x = w + (float)t;
      const float a = t < n ? Am1[t] : 0.f;
      const float b = t >= 1 ? Am1[t - 1] : 0.f;
      B[t] = t <= n ? (x * a + ((float)(n + 1) - x) * b) / (float)n : 0.f;
    }
#pragma unroll
    for (int t = 0; t <= P; ++t) A[t] = B[t];
  }
  // A = M_P, Am1 = M_{P-1}, Am2 = M_{P-2} (for P = 4: M_2 from the start)
#pragma unroll
  for (int t = 0; t < P; ++t) {
    M[t] = A[t];
    dM[t] = (t < P - 1 ? Am1[t] : 0.f) - (t >= 1 ? Am1[t - 1] : 0.f);
    const float c0 = t < P - 2 ? Am2[t] : 0.f, c1 = (t >= 1 && t - 1 < P - 2) ? Am2[t - 1] : 0.f;
    const float c2 = (t >= 2 && t - 2 < P - 2) ? Am2[t - 2] : 0.f;
    d2M[t] = c0 - 2.f * c1 + c2;
  }
}

// fractional grid coordinate of a point C + x (C a wrapped cluster centre as a double-float, x
// the cluster-local coordinate) along d: u = K (C + x) / L, split into base = floor(u) and
// w = u - base, both exact to the FP32 rounding of w
__device__ __forceinline__ void grid_coord(const SysConsts& sc, float2 C, float x, int d, int* base, float* w) {
  df s = two_sum(C.x, x);
  s = fast_two_sum(s.hi, s.lo + C.y);
  const float p = s.hi * sc.pme_kl[d].x;
  const float e = fmaf(s.hi, sc.pme_kl[d].x, -p) + fmaf(s.hi, sc.pme_kl[d].y, s.lo * sc.pme_kl[d].x);
  float b = floorf(p);
  float ww = (p - b) + e;
  if (ww < 0.f) {
    b -= 1.f;
    ww += 1.f;
  } else if (ww >= 1.f) {
    b += 1.f;
    ww -= 1.f;
  }
  *base = (int)b;
  *w = fminf(fmaxf(ww, 0.f), 0.99999994f);
}

__device__ __forceinline__ int wrap(int i, int K) {
  i %= K;
  return i < 0 ? i + K : i;
}

// splines of one slot at bead n: grid indices ix[d][t] and M, dM (scaled by K/L), d2M (by (K/L)^2)
template <int P>
__device__ __forceinline__ void slot_splines(const SysConsts& sc, const PathDev& P_, int n, int s, int (*ix)[P],
                                             float (*M)[P], float (*dM)[P], float (*d2M)[P]) {
  const float4 xl = P_.xq[(size_t)n * P_.Qpad + s];
  const int c = s / kCL;
  const float xv[3] = {xl.x, xl.y, xl.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int b;
    float w;
    grid_coord(sc, P_.cwdf[3 * c + d], xv[d], d, &b, &w);
    spline<P>(w, M[d], dM[d], d2M[d]);
    const float kl = sc.pme_kl[d].x;
#pragma unroll
    for (int t = 0; t < P; ++t) {
      ix[d][t] = wrap(b - t, sc.pme_K[d]);
      dM[d][t] *= kl;
      d2M[d][t] *= kl * kl;
    }
  }
}

// spreads the charges (DERIV = 0) or the charge grid's derivative along eta (DERIV = 1) of every
// slot of bead n onto grid[n] (fixed point); grid: (slots, beads, paths)
template <int P, int DERIV>
__global__ void __launch_bounds__(kRedBlock) k_pme_spread(SysConsts sc, const PathDev* __restrict__ paths) {
  const PathDev& Pd = paths[blockIdx.z];
  const int n = blockIdx.y, s = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_pass = DERIV ? Pd.n_hvp : Pd.n_force;
  if (n >= n_pass || s >= __ldg(&Pd.meta[0]) * kCL) return;
  const int a = Pd.perm[s];
  if (a < 0) return;
  const float q = (float)sc.qs[a];
  if (q == 0.f) return;
  int ix[3][P];
  float M[3][P], dM[3][P], d2M[3][P];
  slot_splines<P>(sc, Pd, n, s, ix, M, dM, d2M);
  float eta[3] = {0.f, 0.f, 0.f};
  if (DERIV) {
    const float4 e = Pd.eta32[(size_t)n * Pd.Qpad + s];
    eta[0] = e.x;
    eta[1] = e.y;
    eta[2] = e.z;
  }
  const int K1 = sc.pme_K[1], K2 = sc.pme_K[2];
  unsigned long long* g = Pd.pme_q + (size_t)n * sc.pme_nk;
#pragma unroll
  for (int t0 = 0; t0 < P; ++t0)
#pragma unroll
    for (int t1 = 0; t1 < P; ++t1) {
      const size_t row = ((size_t)ix[0][t0] * K1 + ix[1][t1]) * K2;
#pragma unroll
      for (int t2 = 0; t2 < P; ++t2) {
        float v;
        if (DERIV)
          v = q * (dM[0][t0] * M[1][t1] * M[2][t2] * eta[0] + M[0][t0] * dM[1][t1] * M[2][t2] * eta[1] +
                   M[0][t0] * M[1][t1] * dM[2][t2] * eta[2]);
        else
          v = q * M[0][t0] * M[1][t1] * M[2][t2];
        atomicAdd(g + row + ix[2][t2], (unsigned long long)__float2ll_rn(v * kGridFixF));
      }
    }
}

// forces (MODE 0: F_i = -q_i sum_k grad M_i(k) phi(k)) or H eta (MODE 1) of every slot, added
// to the fixed-point j-side sums; grid: (slots, beads, paths)
#ifndef MOP_GATHER_MINB
#define MOP_GATHER_MINB 3   // H eta gather: 3 blocks of 256 per SM (80 registers); the force gather runs 4
#endif
template <int P, int MODE>
__global__ void __launch_bounds__(kRedBlock, MODE ? MOP_GATHER_MINB : 4) k_pme_gather(SysConsts sc, const PathDev* __restrict__ paths) {
  const PathDev& Pd = paths[blockIdx.z];
  const int n = blockIdx.y, s = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_pass = MODE ? Pd.n_hvp : Pd.n_force;
  if (n >= n_pass || s >= __ldg(&Pd.meta[0]) * kCL) return;
  const int a = Pd.perm[s];
  if (a < 0) return;
  const float q = (float)sc.qs[a];
  if (q == 0.f) return;
  int ix[3][P];
  float M[3][P], dM[3][P], d2M[3][P];
  slot_splines<P>(sc, Pd, n, s, ix, M, dM, d2M);
  float eta[3] = {0.f, 0.f, 0.f};
  if (MODE) {
    const float4 e = Pd.eta32[(size_t)n * Pd.Qpad + s];
    eta[0] = e.x;
    eta[1] = e.y;
    eta[2] = e.z;
  }
  const int K1 = sc.pme_K[1], K2 = sc.pme_K[2];
  const float* phi = Pd.pme_phi + (size_t)n * sc.pme_nk;
  const float* phd = MODE ? Pd.pme_phd + (size_t)n * sc.pme_nk : nullptr;
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int t0 = 0; t0 < P; ++t0)
#pragma unroll
    for (int t1 = 0; t1 < P; ++t1) {
      const size_t row = ((size_t)ix[0][t0] * K1 + ix[1][t1]) * K2;
#pragma unroll
      for (int t2 = 0; t2 < P; ++t2) {
        const float p = phi[row + ix[2][t2]];
        const float g0 = dM[0][t0] * M[1][t1] * M[2][t2], g1 = M[0][t0] * dM[1][t1] * M[2][t2],
                    g2 = M[0][t0] * M[1][t1] * dM[2][t2];
        if (MODE == 0) {
          acc[0] = fmaf(g0, p, acc[0]);
          acc[1] = fmaf(g1, p, acc[1]);
          acc[2] = fmaf(g2, p, acc[2]);
        } else {
          const float pd = phd[row + ix[2][t2]];
          // (eta . grad) grad of M0 M1 M2 at this point
          const float h00 = d2M[0][t0] * M[1][t1] * M[2][t2], h11 = M[0][t0] * d2M[1][t1] * M[2][t2],
                      h22 = M[0][t0] * M[1][t1] * d2M[2][t2];
          const float h01 = dM[0][t0] * dM[1][t1] * M[2][t2], h02 = dM[0][t0] * M[1][t1] * dM[2][t2],
                      h12 = M[0][t0] * dM[1][t1] * dM[2][t2];
          acc[0] += (h00 * eta[0] + h01 * eta[1] + h02 * eta[2]) * p + g0 * pd;
          acc[1] += (h01 * eta[0] + h11 * eta[1] + h12 * eta[2]) * p + g1 * pd;
          acc[2] += (h02 * eta[0] + h12 * eta[1] + h22 * eta[2]) * p + g2 * pd;
        }
      }
    }
  // forces: -q grad E; H eta: +q (...)
  const float sgn = MODE ? q : -q;
  unsigned long long* dst = Pd.jacc + 3 * ((size_t)n * Pd.Qpad + s);
#pragma unroll
  for (int d = 0; d < 3; ++d) atomicAdd(dst + d, (unsigned long long)__float2ll_rn(sgn * acc[d] * kFixScale));
}

// ---- order-4 spreading: one warp per (cluster, bead) ------------------------------------------
// Lane l < 24 evaluates the splines of atom l / 3 of the cluster along dimension l % 3 once; the
// stencil is then walked two atoms at a time with lane = 16 h + 4 t1 + t2 (atom 2 p + h), each lane
// taking the four points t0 = 0..3 of its (t1, t2) column.  The four lanes of a (t0, t1) row add
// to consecutive grid words, so their atomics share memory sectors (about half the time of one
// thread per atom walking its 64 points).  Gathering stays one thread per atom: there the
// overlapping stencils of a warp hit in L1 and cross-lane traffic only costs.
struct Spl4 {
  int b;                 // base grid index along this lane's dimension
  float M[4], dM[4];     // values and d/dx (scaled by K/L)
  float q, e;            // sqrt(f) q of the atom (0: padding), eta along this dimension
};

template <bool ETA>
__device__ __forceinline__ void lane_spline4(const SysConsts& sc, const PathDev& Pd, int n, int c, int lane,
                                             Spl4& S) {
  S.b = 0;
  S.q = S.e = 0.f;
#pragma unroll
  for (int t = 0; t < 4; ++t) S.M[t] = S.dM[t] = 0.f;
  if (lane >= 24) return;
  const int a = lane / 3, d = lane - 3 * a;
  const size_t k = (size_t)n * Pd.Qpad + c * kCL + a;
  const float4 xl = Pd.xq[k];
  const float x = d == 0 ? xl.x : (d == 1 ? xl.y : xl.z);
  float w, d2[4];
  grid_coord(sc, Pd.cwdf[3 * c + d], x, d, &S.b, &w);
  spline<4>(w, S.M, S.dM, d2);
  const float kl = sc.pme_kl[d].x;
#pragma unroll
  for (int t = 0; t < 4; ++t) S.dM[t] *= kl;
  S.q = xl.w;   // padding slots carry 0
  if (ETA) {
    const float4 e = Pd.eta32[k];
    S.e = d == 0 ? e.x : (d == 1 ? e.y : e.z);
  }
}

__device__ __forceinline__ float sel4(const float (&v)[4], int t) {
  return t == 0 ? v[0] : (t == 1 ? v[1] : (t == 2 ? v[2] : v[3]));
}

// atom A's splines as this lane uses them: the whole t0 row of dimension 0, the (t1, t2) entries
struct Walk4 {
  int b0, r12;       // base along 0; grid offset of this lane's (t1, t2) column
  float q, e0, e1, e2;
  float M0[4], dM0[4];
  float m1, dm1, m2, dm2;
};

template <bool ETA>
__device__ __forceinline__ void walk4(const SysConsts& sc, const Spl4& S, int A, int t1, int t2, Walk4& W) {
  const unsigned full = 0xffffffffu;
  const int s0 = 3 * A, s1 = s0 + 1, s2 = s0 + 2;
  float M1[4], M2[4], dM1[4], dM2[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    W.M0[t] = __shfl_sync(full, S.M[t], s0);
    W.dM0[t] = __shfl_sync(full, S.dM[t], s0);
    M1[t] = __shfl_sync(full, S.M[t], s1);
    dM1[t] = __shfl_sync(full, S.dM[t], s1);
    M2[t] = __shfl_sync(full, S.M[t], s2);
    dM2[t] = __shfl_sync(full, S.dM[t], s2);
  }
  W.m1 = sel4(M1, t1);
  W.dm1 = sel4(dM1, t1);
  W.m2 = sel4(M2, t2);
  W.dm2 = sel4(dM2, t2);
  W.q = __shfl_sync(full, S.q, s0);
  if (ETA) {
    W.e0 = __shfl_sync(full, S.e, s0);
    W.e1 = __shfl_sync(full, S.e, s1);
    W.e2 = __shfl_sync(full, S.e, s2);
  }
  W.b0 = __shfl_sync(full, S.b, s0);
  const int b1 = __shfl_sync(full, S.b, s1), b2 = __shfl_sync(full, S.b, s2);
  W.r12 = wrap(b1 - t1, sc.pme_K[1]) * sc.pme_K[2] + wrap(b2 - t2, sc.pme_K[2]);
}

template <int DERIV>
__global__ void __launch_bounds__(128) k_pme_spread4(SysConsts sc, const PathDev* __restrict__ paths) {
  const PathDev& Pd = paths[blockIdx.z];
  const int n = blockIdx.y, lane = threadIdx.x & 31;
  const int c = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int n_pass = DERIV ? Pd.n_hvp : Pd.n_force;
  if (n >= n_pass || c >= __ldg(&Pd.meta[0])) return;   // whole warps
  Spl4 S;
  lane_spline4<DERIV == 1>(sc, Pd, n, c, lane, S);
  const int h = lane >> 4, t1 = (lane >> 2) & 3, t2 = lane & 3;
  const size_t plane = (size_t)sc.pme_K[1] * sc.pme_K[2];
  unsigned long long* g = Pd.pme_q + (size_t)n * sc.pme_nk;
#pragma unroll 1
  for (int p = 0; p < 4; ++p) {
    Walk4 W;
    walk4<DERIV == 1>(sc, S, 2 * p + h, t1, t2, W);
    if (W.q == 0.f) continue;
#pragma unroll
    for (int t0 = 0; t0 < 4; ++t0) {
      float v;
      if (DERIV)
        v = W.q * (W.dM0[t0] * W.m1 * W.m2 * W.e0 + W.M0[t0] * (W.dm1 * W.m2 * W.e1 + W.m1 * W.dm2 * W.e2));
      else
        v = W.q * W.M0[t0] * W.m1 * W.m2;
      atomicAdd(g + wrap(W.b0 - t0, sc.pme_K[0]) * plane + W.r12,
                (unsigned long long)__float2ll_rn(v * kGridFixF));
    }
  }
}

template <int P>
cudaError_t run_pme(const SysConsts& sc, const PathDev* d_paths, const PathDev* h_paths, int n_paths, int max_beads,
                    int mode, PmePlans& plans, Launch L, std::string* err) {
  int max_qpad = 0;
  for (int p = 0; p < n_paths; ++p) max_qpad = std::max(max_qpad, h_paths[p].Qpad);
  const dim3 sgrid((max_qpad + kRedBlock - 1) / kRedBlock, max_beads, n_paths);
  for (int p = 0; p < n_paths; ++p) {
    const PathDev& D = h_paths[p];
    const int beads = mode ? D.n_hvp : D.n_force;
    if (beads <= 0) continue;
    cudaError_t e = cudaMemsetAsync(D.pme_q, 0, sizeof(unsigned long long) * sc.pme_nk * beads, L.st);
    if (e != cudaSuccess) return e;
  }
  int max_clu = 0;
  for (int p = 0; p < n_paths; ++p) max_clu = std::max(max_clu, h_paths[p].n_clu);
  const dim3 wgrid((max_clu + 3) / 4, max_beads, n_paths);
  if (P == 4) {
    if (mode == 0) k_pme_spread4<0><<<wgrid, 128, 0, L.st>>>(sc, d_paths);
    else k_pme_spread4<1><<<wgrid, 128, 0, L.st>>>(sc, d_paths);
  } else {
    if (mode == 0) k_pme_spread<P, 0><<<sgrid, kRedBlock, 0, L.st>>>(sc, d_paths);
    else k_pme_spread<P, 1><<<sgrid, kRedBlock, 0, L.st>>>(sc, d_paths);
  }
  ++*L.counter;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!plans.ready) {
    if (err) *err = "no FFT plan for this grid (evaluate once without stream capture first)";
    return cudaErrorNotReady;
  }
  for (int p = 0; p < n_paths; ++p) {
    const PathDev& D = h_paths[p];
    const int beads = mode ? D.n_hvp : D.n_force;
    if (beads <= 0) continue;
    e = launch_fft_convolve(sc, plans.ax, D.pme_q, D.pme_c, mode ? D.pme_phd : D.pme_phi, beads,
                            mode == 0 ? D.pme_e : nullptr, L);
    if (e != cudaSuccess) return e;
  }
  if (mode == 0) k_pme_gather<P, 0><<<sgrid, kRedBlock, 0, L.st>>>(sc, d_paths);
  else k_pme_gather<P, 1><<<sgrid, kRedBlock, 0, L.st>>>(sc, d_paths);
  ++*L.counter;
  return cudaGetLastError();
}

}  // namespace

PmePlans* pme_plans_create() { return new PmePlans(); }
void pme_plans_destroy(PmePlans* p) { delete p; }

// makes the twiddle tables of the grid once (never inside a stream capture); any bead count
cudaError_t pme_plans_ensure(const SysConsts& sc, PmePlans* plans, int beads, std::string* err) {
  (void)beads;
  if (plans->ready) return cudaSuccess;
  for (int d = 0; d < 3; ++d) {
    cudaError_t e = fft_axis_make(sc.pme_K[d], plans->tw[d], &plans->ax[d]);
    if (e != cudaSuccess) {
      if (err) *err = "FFT tables of the SPME grid";
      return e == cudaErrorInvalidValue ? cudaErrorInvalidValue : cudaErrorMemoryAllocation;
    }
  }
  plans->ready = true;
  return cudaSuccess;
}

cudaError_t launch_pme(const SysConsts& sc, const PathDev* d_paths, const PathDev* h_paths, int n_paths,
                       int max_beads, int mode, PmePlans* plans, Launch L, std::string* err) {
  switch (sc.pme_order) {
    case 4: return run_pme<4>(sc, d_paths, h_paths, n_paths, max_beads, mode, *plans, L, err);
    case 5: return run_pme<5>(sc, d_paths, h_paths, n_paths, max_beads, mode, *plans, L, err);
    case 6: return run_pme<6>(sc, d_paths, h_paths, n_paths, max_beads, mode, *plans, L, err);
    case 7: return run_pme<7>(sc, d_paths, h_paths, n_paths, max_beads, mode, *plans, L, err);
    default: return run_pme<8>(sc, d_paths, h_paths, n_paths, max_beads, mode, *plans, L, err);
  }
}

}  // namespace mop
