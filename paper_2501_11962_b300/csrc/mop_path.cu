// Elementwise kernels of the path: bonded terms and eta (after the force pass), bonded HVP and
// the path gradient (after the HVP pass), the metadynamics bias, the deterministic V_eff
// reduction, and the path-dynamics integrator.
//
// Paper: the seven PMD kernels of Sec. 2.1 (Fig. 2): eta^n = R^{n+1} - R^n - L^n (kernel 1),
// the effective forces of Eqs. 5, 6, 7 (kernels 4-6), the spring energy (kernel 7); the bias of
// Sec. 1.2 with the CV of Eq. 8; the dynamics of Eq. 4.  The exact gradient written here,
//   G^1 = -F^1 - K eta^1 + H eta^1 / 2,   G^n = K eta^{n-1} - K eta^n + H eta^n / 2,
//   G^N = K eta^{N-1},
// equals minus the effective force of Eqs. 5-7 once the FD term is replaced by -H eta / 2
// (K_i L^n_i = F^n_i / 2 turns K eta^{n-1} into K (R^n - R^{n-1}) - F^{n-1} / 2).
#include "mop_host.h"

namespace mop {
namespace {

// ------------------------------------------------------------------------------------------
// forward-mode dual numbers (value, tangent) for the bonded Hessian-vector product

template <class R> struct Dl {
  R v, d;
};
template <class R> __device__ __forceinline__ Dl<R> operator+(Dl<R> a, Dl<R> b) { return {a.v + b.v, a.d + b.d}; }
template <class R> __device__ __forceinline__ Dl<R> operator-(Dl<R> a, Dl<R> b) { return {a.v - b.v, a.d - b.d}; }
template <class R> __device__ __forceinline__ Dl<R> operator-(Dl<R> a) { return {-a.v, -a.d}; }
template <class R> __device__ __forceinline__ Dl<R> operator*(Dl<R> a, Dl<R> b) {
  return {a.v * b.v, a.v * b.d + a.d * b.v};
}
template <class R> __device__ __forceinline__ Dl<R> operator*(R s, Dl<R> a) { return {s * a.v, s * a.d}; }
template <class R> __device__ __forceinline__ Dl<R> operator/(Dl<R> a, Dl<R> b) {
  const R iv = R(1) / b.v;
  return {a.v * iv, (a.d - a.v * iv * b.d) * iv};
}
template <class R> __device__ __forceinline__ Dl<R> dsqrt(Dl<R> a) {
  const R s = sqrt(a.v);
  return {s, a.d / (R(2) * s)};
}
template <class R> __device__ __forceinline__ Dl<R> dacos(Dl<R> a) {
  return {acos(a.v), -a.d / sqrt(R(1) - a.v * a.v)};
}
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float dacos(float a) { return acosf(a); }
__device__ __forceinline__ double dacos(double a) { return acos(a); }
template <class R> __device__ __forceinline__ R cst(double c) { return (R)c; }

template <class T, class R> struct Mk {
  static __device__ __forceinline__ T c(R v) { return v; }
};
template <class R> struct Mk<Dl<R>, R> {
  static __device__ __forceinline__ Dl<R> c(R v) { return {v, R(0)}; }
};

// harmonic bond k/2 (|d| - r0)^2, d = x_i - x_j: force on the atom with the given role
template <class T, class R>
__device__ __forceinline__ void bond_force(const T* d, R r0, R k, int role, T* f, R* U) {
  const T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const T r = dsqrt(r2);
  const T dr = r - Mk<T, R>::c(r0);
  const T s = (-k) * (dr / r);
  const R sg = role == 0 ? R(1) : R(-1);
  for (int c = 0; c < 3; ++c) f[c] = sg * (s * d[c]);
  if (U) {
    const T u = dr * dr;
    if constexpr (sizeof(T) == sizeof(R)) *U = R(0.5) * k * u;
  }
}

// harmonic angle k/2 (theta - theta0)^2 at vertex j; p = x_i - x_j, q = x_k - x_j
template <class T, class R>
__device__ __forceinline__ void angle_force(const T* p, const T* q, R th0, R k, int role, T* f, R* U) {
  const T pp = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
  const T qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  const T pq = p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
  const T inpq = Mk<T, R>::c(R(1)) / (dsqrt(pp) * dsqrt(qq));
  const T c = pq * inpq;
  const T th = dacos(c);
  const T dth = th - Mk<T, R>::c(th0);
  const T sn = dsqrt(Mk<T, R>::c(R(1)) - c * c);
  const T G = k * (dth / sn);   // -dU/dcos
  const T cp = c / pp, cq = c / qq;
  for (int m = 0; m < 3; ++m) {
    const T dcp = q[m] * inpq - cp * p[m];
    const T dcq = p[m] * inpq - cq * q[m];
    const T fi = G * dcp, fk = G * dcq;
    f[m] = role == 0 ? fi : (role == 2 ? fk : -(fi + fk));
  }
  if (U) {
    if constexpr (sizeof(T) == sizeof(R)) *U = R(0.5) * k * dth * dth;
  }
}

// minimum-image difference x_a - x_b of bead n in the caller's coordinates
template <class R>
__device__ __forceinline__ void mi_diff(const SysConsts& sc, const PathDev& P, int n, int a, int b, R* d) {
  const size_t base = (size_t)n * 3 * P.Q;
  if (P.x64) {
    for (int c = 0; c < 3; ++c) {
      double v = P.x64[base + 3 * (size_t)a + c] - P.x64[base + 3 * (size_t)b + c];
      v -= sc.L[c] * rint(v * sc.invL[c]);
      d[c] = (R)v;
    }
    return;
  }
  for (int c = 0; c < 3; ++c) {
    const float xa = P.x32[base + 3 * (size_t)a + c], xb = P.x32[base + 3 * (size_t)b + c];
    float v = xa - xb;   // exact when both lie in the same periodic image
    if (fabsf(v) > sc.halfLf[c]) {
      // across images, in FP32 only (the FP64 pipe is slow and a warp takes this branch
      // whenever any lane does): the exact difference w = xa - xb as a double-float, minus
      // k L with L = (Lf, Llo) and k Lf formed exactly by an FMA
      const df w = two_sum(xa, -xb);
      const float k = rintf(w.hi * sc.invLf[c]);
      const float p = k * sc.Lf[c];
      const df r = df_add(w, df{-p, -fmaf(k, sc.Lf[c], -p)});
      v = r.hi + (r.lo - k * sc.Llo[c]);
    }
    d[c] = (R)v;
  }
}

template <class R>
__device__ __forceinline__ void eta_of(const PathDev& P, int n, int atom, R* e) {
  const size_t k = (size_t)n * P.Qpad + P.slot[atom];
  if (sizeof(R) == 4) {
    const float4 v = P.eta32[k];
    e[0] = (R)v.x;
    e[1] = (R)v.y;
    e[2] = (R)v.z;
  } else {
    e[0] = (R)P.eta[3 * k];
    e[1] = (R)P.eta[3 * k + 1];
    e[2] = (R)P.eta[3 * k + 2];
  }
}

// Bonded force on atom a at bead n, accumulated in FP64; U (if non-NULL) gets the energy of
// the terms for which a has role 0 (so that every term is counted once).
template <class R> __device__ __forceinline__ void term_params(const SysConsts& sc, int t, R* a, R* b);
template <> __device__ __forceinline__ void term_params<float>(const SysConsts& sc, int t, float* a, float* b) {
  const float2 v = sc.incpf[t];
  *a = v.x;
  *b = v.y;
}
template <> __device__ __forceinline__ void term_params<double>(const SysConsts& sc, int t, double* a, double* b) {
  const double2 v = sc.incp[t];
  *a = v.x;
  *b = v.y;
}

template <class R, class A, class U_t>
__device__ void bonded_force(const SysConsts& sc, const PathDev& P, int a, int n, A* F, U_t* U) {
  for (int t = sc.inc_off[a]; t < sc.inc_off[a + 1]; ++t) {
    const int4 in = sc.inc[t];
    R pr0, pr1;
    term_params<R>(sc, t, &pr0, &pr1);
    const int kind = in.x & 3, role = in.x >> 2;
    R f[3];
    R u = R(0);
    if (kind == 0) {
      R d[3];
      mi_diff<R>(sc, P, n, in.y, in.z, d);
      bond_force<R, R>(d, pr0, pr1, role, f, U && role == 0 ? &u : nullptr);
    } else {
      R p[3], q[3];
      mi_diff<R>(sc, P, n, in.y, in.z, p);
      mi_diff<R>(sc, P, n, in.w, in.z, q);
      angle_force<R, R>(p, q, pr0, pr1, role, f, U && role == 0 ? &u : nullptr);
    }
    F[0] += (A)f[0];
    F[1] += (A)f[1];
    F[2] += (A)f[2];
    if (U && role == 0) *U += u;
  }
}

// Bonded H eta on atom a at bead n: adjoint (dual numbers) or central difference with eps.
template <class R, bool FD, class A>
__device__ void bonded_hvp(const SysConsts& sc, const PathDev& P, int a, int n, double eps, A* H) {
  for (int t = sc.inc_off[a]; t < sc.inc_off[a + 1]; ++t) {
    const int4 in = sc.inc[t];
    R pr0, pr1;
    term_params<R>(sc, t, &pr0, &pr1);
    const int kind = in.x & 3, role = in.x >> 2;
    // relative vectors and their tangents (differences of eta)
    R v1[3], v2[3], t1[3], t2[3];
    R ei[3], ej[3], ek[3];
    eta_of<R>(P, n, in.y, ei);
    eta_of<R>(P, n, in.z, ej);
    mi_diff<R>(sc, P, n, in.y, in.z, v1);
    for (int c = 0; c < 3; ++c) t1[c] = ei[c] - ej[c];
    if (kind == 1) {
      eta_of<R>(P, n, in.w, ek);
      mi_diff<R>(sc, P, n, in.w, in.z, v2);
      for (int c = 0; c < 3; ++c) t2[c] = ek[c] - ej[c];
    }
    if (!FD) {
      Dl<R> d1[3], d2[3], f[3];
      for (int c = 0; c < 3; ++c) {
        d1[c] = {v1[c], t1[c]};
        d2[c] = {kind == 1 ? v2[c] : R(0), kind == 1 ? t2[c] : R(0)};
      }
      if (kind == 0) bond_force<Dl<R>, R>(d1, pr0, pr1, role, f, nullptr);
      else angle_force<Dl<R>, R>(d1, d2, pr0, pr1, role, f, nullptr);
      for (int c = 0; c < 3; ++c) H[c] -= (A)f[c].d;   // H eta = -d/dt F(x + t eta)
    } else {
      R fp[3], fm[3], a1[3], a2[3];
      const R e = (R)eps;
      for (int s = 0; s < 2; ++s) {
        const R sg = s == 0 ? e : -e;
        for (int c = 0; c < 3; ++c) {
          a1[c] = v1[c] + sg * t1[c];
          a2[c] = kind == 1 ? v2[c] + sg * t2[c] : R(0);
        }
        R* f = s == 0 ? fp : fm;
        if (kind == 0) bond_force<R, R>(a1, pr0, pr1, role, f, nullptr);
        else angle_force<R, R>(a1, a2, pr0, pr1, role, f, nullptr);
      }
      if (sizeof(A) == 4) {
        const R inv2e = R(0.5) / (R)eps;
        for (int c = 0; c < 3; ++c) H[c] -= (A)((fp[c] - fm[c]) * inv2e);
      } else {
        for (int c = 0; c < 3; ++c) H[c] -= (A)(((double)fp[c] - (double)fm[c]) / (2.0 * eps));
      }
    }
  }
}

// E1: F^n = F_nonbonded + F_bonded, eta^n = R^{n+1} - R^n - c F^n (FP64), bonded energy of bead 1
template <class R>
__global__ void __launch_bounds__(kRedBlock) k_e1(SysConsts sc, const PathDev* __restrict__ paths, int n_paths,
                                                  double* e_bond, int nbx) {
  __shared__ double sh[32];
  const int p = blockIdx.z, n = blockIdx.y;
  const PathDev& P = paths[p];
  if (n >= P.n_force) return;   // whole block; only bead-1 blocks write energy partials
  const int a = blockIdx.x * blockDim.x + threadIdx.x;   // caller order: molecules are contiguous
  double eb = 0.0;
  if (a < P.Q) {
    const int s = P.slot[a];
    const size_t k = (size_t)n * P.Qpad + s;
    double F[3] = {0.0, 0.0, 0.0}, e[3] = {0.0, 0.0, 0.0};
    {
      F[0] = P.Fnb[3 * k];
      F[1] = P.Fnb[3 * k + 1];
      F[2] = P.Fnb[3 * k + 2];
      bonded_force<R, double, double>(sc, P, a, n, F, n == 0 ? &eb : nullptr);
      if (P.N > 1) {
        const size_t b0 = (size_t)n * 3 * P.Q + 3 * (size_t)a, b1 = b0 + 3 * (size_t)P.Q;
        const double c = sc.cL[a];
        for (int d = 0; d < 3; ++d) {
          const double x0 = P.x64 ? P.x64[b0 + d] : (double)P.x32[b0 + d];
          const double x1 = P.x64 ? P.x64[b1 + d] : (double)P.x32[b1 + d];
          e[d] = (x1 - x0) - c * F[d];
        }
        if (sc.hvp_mode == 1) {
          const double nrm = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
          atomicMax(&P.etamax[n], __float_as_uint(__double2float_ru(nrm)));
        }
      }
    }
    P.F[3 * k] = F[0];
    P.F[3 * k + 1] = F[1];
    P.F[3 * k + 2] = F[2];
    if (P.N > 1) {
      P.eta[3 * k] = e[0];
      P.eta[3 * k + 1] = e[1];
      P.eta[3 * k + 2] = e[2];
      P.eta32[k] = make_float4((float)e[0], (float)e[1], (float)e[2], 0.f);
    }
  }
  if (n == 0) {
    const double tot = block_sum<kRedBlock>(eb, sh);
    if (threadIdx.x == 0) e_bond[(size_t)p * nbx + blockIdx.x] = tot;
  }
}

// E2: bonded H eta, H eta total, path gradient (caller order), spring energy
template <class R, bool FD>
__global__ void __launch_bounds__(kRedBlock) k_e2(SysConsts sc, const PathDev* __restrict__ paths, int n_paths,
                                                  double* e_spring, int nbx, int maxN, int n_begin) {
  __shared__ double sh[32];
  const int p = blockIdx.z, n = n_begin + blockIdx.y;
  const PathDev& P = paths[p];
  double* part = e_spring + ((size_t)p * maxN + n) * nbx + blockIdx.x;
  if (n >= P.N) {
    if (threadIdx.x == 0) *part = 0.0;
    return;
  }
  const int a = blockIdx.x * blockDim.x + threadIdx.x;   // caller order
  double es = 0.0;
  if (a < P.Q) {
    const int s = P.slot[a];
    const size_t k = (size_t)n * P.Qpad + s;
    {
      const double K = sc.Kspr[a];
      double g[3] = {0.0, 0.0, 0.0};
      if (n == 0)
        for (int c = 0; c < 3; ++c) g[c] -= P.F[3 * (size_t)s + c];
      if (n > 0) {
        const size_t km = k - P.Qpad;
        for (int c = 0; c < 3; ++c) g[c] += K * P.eta[3 * km + c];
      }
      if (n < P.N - 1) {
        double H[3] = {P.Hnb[3 * k], P.Hnb[3 * k + 1], P.Hnb[3 * k + 2]};
        double eps = 0.0;
        if (FD) {
          const float mx = __uint_as_float(P.etamax[n]);
          eps = mx > 0.f ? sc.fd_h / (double)mx : sc.fd_h;
          eps = (double)(R)eps;   // the pair kernel used the same eps in its own precision
        }
        bonded_hvp<R, FD, double>(sc, P, a, n, eps, H);
        double e2 = 0.0;
        for (int c = 0; c < 3; ++c) {
          const double e = P.eta[3 * k + c];
          P.Heta[3 * k + c] = H[c];
          g[c] += -K * e + 0.5 * H[c];
          e2 += e * e;
        }
        es = 0.5 * K * e2;
      }
      double* G = P.grad + 3 * ((size_t)n * P.Q + a);
      G[0] = g[0];
      G[1] = g[1];
      G[2] = g[2];
    }
  }
  const double tot = block_sum<kRedBlock>(es, sh);
  if (threadIdx.x == 0) *part = tot;
}

// ------------------------------------------------------------------------------------------
// mixed precision (MOP_PREC_MIXED): FP32 arithmetic with double-float where cancellation needs
// more than FP32.  F^n = F_nonbonded (double-float from the pair kernel) + F_bonded;
// eta^n = (R^{n+1} - R^n) - c F^n in double-float (the difference of nearly equal terms when
// the path is close to a solution of Eq. 1), stored rounded to FP32; bonded energy of bead 1.
#ifndef MOP_E1_MINB
#define MOP_E1_MINB 6   // 40 registers
#endif
#ifndef MOP_E2_MINB
#define MOP_E2_MINB 4   // 64 registers: 4 blocks of 256 per SM instead of 3 (E2 0.68 -> 0.59 ms at 150k atoms x 64 beads)
#endif
#if MOP_E1_MINB > 0
#define MOP_E1_BOUNDS __launch_bounds__(kRedBlock, MOP_E1_MINB)
#else
#define MOP_E1_BOUNDS __launch_bounds__(kRedBlock)
#endif
#if MOP_E2_MINB > 0
#define MOP_E2_BOUNDS __launch_bounds__(kRedBlock, MOP_E2_MINB)
#else
#define MOP_E2_BOUNDS __launch_bounds__(kRedBlock)
#endif
__global__ void MOP_E1_BOUNDS k_e1_mixed(SysConsts sc, const PathDev* __restrict__ paths, int n_paths,
                                                        double* e_bond, int nbx) {
  __shared__ double shw[kRedBlock / 32];
  const int p = blockIdx.z, n = blockIdx.y;
  const PathDev& P = paths[p];
  if (n >= P.n_force) return;   // whole block; only bead-1 blocks write energy partials
  const int a = blockIdx.x * blockDim.x + threadIdx.x;   // caller order: molecules are contiguous
  float eb = 0.f;
  unsigned nbits = 0u;
  if (a < P.Q) {
    const int s = P.slot[a];
    const size_t k = (size_t)n * P.Qpad + s;
    const float2* Fnb = reinterpret_cast<const float2*>(P.Fnb) + 3 * k;
    float2* Fo = reinterpret_cast<float2*>(P.F) + 3 * k;
    df F[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    float4 ef = make_float4(0.f, 0.f, 0.f, 0.f), efl = ef;
    {
      float Fb[3] = {0.f, 0.f, 0.f};
      bonded_force<float, float, float>(sc, P, a, n, Fb, n == 0 ? &eb : nullptr);
      for (int c = 0; c < 3; ++c) {
        F[c] = df_add_f(df{Fnb[c].x, Fnb[c].y}, Fb[c]);
        if (P.jacc) F[c] = df_add(F[c], fix_to_df((long long)P.jacc[3 * k + c]));   // j-side sums
      }
      if (P.N > 1) {
        const size_t b0 = (size_t)n * 3 * P.Q + 3 * (size_t)a, b1 = b0 + 3 * (size_t)P.Q;
        const float2 cc = sc.c_df[a];
        float e[3], el[3];
        for (int c = 0; c < 3; ++c) {
          const df d = two_sum(P.x32[b1 + c], -P.x32[b0 + c]);   // exact R^{n+1} - R^n
          const df cf = df_mul(df{cc.x, cc.y}, F[c]);
          const df et = df_add(d, df_neg(cf));   // normalised: hi = FP32 rounding of eta
          e[c] = et.hi;
          el[c] = et.lo;
        }
        ef = make_float4(e[0], e[1], e[2], 0.f);
        efl = make_float4(el[0], el[1], el[2], 0.f);
        // max_i |eta_i| per bead: the FD step, and the scale of the half list's j-side sums
        if (sc.hvp_mode == 1 || sc.bl == 1 || sc.bl == 2)
          nbits = __float_as_uint(sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) * 1.000001f);
      }
    }
    for (int c = 0; c < 3; ++c) Fo[c] = make_float2(F[c].hi, F[c].lo);
    if (P.N > 1) {
      P.eta32[k] = ef;
      P.etalo[k] = efl;
    }
  }
  if (sc.hvp_mode == 1 || sc.bl == 1 || sc.bl == 2) {
    // one atomic per warp (all lanes belong to bead n)
    const unsigned mx = __reduce_max_sync(0xffffffffu, nbits);
    if ((threadIdx.x & 31) == 0) atomicMax(&P.etamax[n], mx);
  }
  if (n == 0) {
    const df w = df_warp_sum(df{eb, 0.f});
    if ((threadIdx.x & 31) == 0) shw[threadIdx.x >> 5] = widen(w.hi) + widen(w.lo);
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int k = 0; k < kRedBlock / 32; ++k) tot += shw[k];
      e_bond[(size_t)p * nbx + blockIdx.x] = tot;
    }
  }
}

// H eta (pair part from the HVP kernel + bonded part, FP32), the gradient of Eqs. 5-7 in
// double-float, G^n = K (eta^{n-1} - eta^n) + H eta^n / 2 (- F^1 at bead 1), from the double-float
// eta and F of E1, written as FP64; spring energy summed as double-floats per warp and in FP64
// per block.
template <bool FD>
__global__ void MOP_E2_BOUNDS k_e2_mixed(SysConsts sc, const PathDev* __restrict__ paths, int n_paths,
                                                        double* e_spring, int nbx, int maxN, int n_begin) {
  __shared__ double shw[kRedBlock / 32];
  const int p = blockIdx.z, n = n_begin + blockIdx.y;
  const PathDev& P = paths[p];
  double* part = e_spring + ((size_t)p * maxN + n) * nbx + blockIdx.x;
  if (n >= P.N) {
    if (threadIdx.x == 0) *part = 0.0;
    return;
  }
  const int a = blockIdx.x * blockDim.x + threadIdx.x;   // caller order
  float es = 0.f;
  if (a < P.Q) {
    const int s = P.slot[a];
    const size_t k = (size_t)n * P.Qpad + s;
    {
      const float2 Kv = sc.K_df[a];
      const df K{Kv.x, Kv.y};
      // eta^{n-1} - eta^n as double-floats (eta^{-1} = eta^{N-1} = 0)
      df d[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      if (n > 0) {
        const float4 h = P.eta32[k - P.Qpad], l = P.etalo[k - P.Qpad];
        d[0] = df{h.x, l.x};
        d[1] = df{h.y, l.y};
        d[2] = df{h.z, l.z};
      }
      float H[3] = {0.f, 0.f, 0.f};
      if (n < P.N - 1) {
        const float4 h = P.eta32[k], l = P.etalo[k];
        d[0] = df_add(d[0], df{-h.x, -l.x});
        d[1] = df_add(d[1], df{-h.y, -l.y});
        d[2] = df_add(d[2], df{-h.z, -l.z});
        const float4 hn = reinterpret_cast<const float4*>(P.Hnb)[k];
        H[0] = hn.x;
        H[1] = hn.y;
        H[2] = hn.z;
        if (P.jacc) {   // j-side sums
          const unsigned long long* J = P.jacc + 3 * k;
          for (int c = 0; c < 3; ++c) H[c] += __ll2float_rn((long long)J[c]) * kFixInv;
        }
        double eps = 0.0;
        if (FD) {
          const float mx = __uint_as_float(P.etamax[n]);
          eps = (double)(float)(mx > 0.f ? sc.fd_h / (double)mx : sc.fd_h);
        }
        bonded_hvp<float, FD, float>(sc, P, a, n, eps, H);
        reinterpret_cast<float4*>(P.Heta)[k] = make_float4(H[0], H[1], H[2], 0.f);
        es = 0.5f * Kv.x * (h.x * h.x + h.y * h.y + h.z * h.z);
      }
      df g[3];
      for (int c = 0; c < 3; ++c) g[c] = df_add_f(df_mul(K, d[c]), 0.5f * H[c]);
      if (n == 0) {
        const float2* F1 = reinterpret_cast<const float2*>(P.F) + 3 * (size_t)s;
        for (int c = 0; c < 3; ++c) g[c] = df_add(g[c], df{-F1[c].x, -F1[c].y});
      }
      double* G = P.grad + 3 * ((size_t)n * P.Q + a);
      // hi + lo is exact in FP64; the halves are widened on the integer pipes
      G[0] = widen(g[0].hi) + widen(g[0].lo);
      G[1] = widen(g[1].hi) + widen(g[1].lo);
      G[2] = widen(g[2].hi) + widen(g[2].lo);
    }
  }
  const df w = df_warp_sum(df{es, 0.f});
  if ((threadIdx.x & 31) == 0) shw[threadIdx.x >> 5] = widen(w.hi) + widen(w.lo);
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < kRedBlock / 32; ++k) tot += shw[k];
    *part = tot;
  }
}

// weight of atom a in a group centre: its mass for a mass-weighted CV (centre of mass), else 1
__device__ __forceinline__ double group_weight(const SysConsts& sc, int com, int a) { return com ? sc.mass[a] : 1.0; }

// weighted centre of a group at bead n, each atom unwrapped relative to the group's first atom;
// *W gets the total weight
__device__ void centroid(const SysConsts& sc, const PathDev& P, int n, const int* g, int ng, int com, double* c,
                         double* W) {
  const size_t base = (size_t)n * 3 * P.Q;
  double x0[3], acc[3] = {0.0, 0.0, 0.0}, wt = 0.0;
  for (int d = 0; d < 3; ++d) x0[d] = P.x64 ? P.x64[base + 3 * (size_t)g[0] + d] : (double)P.x32[base + 3 * (size_t)g[0] + d];
  for (int k = 0; k < ng; ++k) {
    const double m = group_weight(sc, com, g[k]);
    for (int d = 0; d < 3; ++d) {
      const double v = P.x64 ? P.x64[base + 3 * (size_t)g[k] + d] : (double)P.x32[base + 3 * (size_t)g[k] + d];
      double w = v - x0[d];
      w -= sc.L[d] * rint(w * sc.invL[d]);
      acc[d] += m * w;
    }
    wt += m;
  }
  for (int d = 0; d < 3; ++d) c[d] = x0[d] + acc[d] / wt;
  *W = wt;
}

// CV q: distance s = |c_A - c_B| (minimum image) of its groups at bead n; u = (c_A - c_B) / s,
// Wa / Wb = the groups' total weights
__device__ double cv_at(const SysConsts& sc, const PathDev& P, int n, int q, double* u, double* Wa, double* Wb) {
  double ca[3], cb[3];
  centroid(sc, P, n, P.gA + P.cv_a[q], P.cv_a[q + 1] - P.cv_a[q], P.cv_com[q], ca, Wa);
  centroid(sc, P, n, P.gB + P.cv_b[q], P.cv_b[q + 1] - P.cv_b[q], P.cv_com[q], cb, Wb);
  double s2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    double w = ca[d] - cb[d];
    w -= sc.L[d] * rint(w * sc.invL[d]);
    u[d] = w;
    s2 += w * w;
  }
  const double s = sqrt(s2);
  for (int d = 0; d < 3; ++d) u[d] /= s;
  return s;
}

// value of CV q of a path: s at bead N, minus s at bead 1 for the end-to-end form (Eq. 8)
__device__ double cv_value(const SysConsts& sc, const PathDev& P, int q, double* uN, double* u1, double* Wa,
                           double* Wb) {
  double S = cv_at(sc, P, P.N - 1, q, uN, Wa, Wb);
  if (P.cv_e2e[q]) S -= cv_at(sc, P, 0, q, u1, Wa, Wb);
  return S;
}

// metadynamics bias (one block per path): V_b = sum_k h_k exp(-sum_q (S_q - c_kq)^2 / (2 w_kq^2))
__global__ void k_bias(SysConsts sc, const PathDev* __restrict__ paths, int n_paths) {
  __shared__ double sh[32];
  __shared__ double sS[kMaxCV], sU[kMaxCV][2][3], sW[kMaxCV][2];
  const PathDev& P = paths[blockIdx.x];
  const int nc = P.n_cv;
  const bool on = P.n_gauss > 0 && nc > 0;
  if (threadIdx.x == 0)
    for (int q = 0; q < nc; ++q) sS[q] = cv_value(sc, P, q, sU[q][0], sU[q][1], &sW[q][0], &sW[q][1]);
  __syncthreads();
  double V = 0.0, dV[kMaxCV] = {0.0, 0.0, 0.0, 0.0};
  if (on)
    for (int k = threadIdx.x; k < P.n_gauss; k += blockDim.x) {
      double z2 = 0.0;
      for (int q = 0; q < nc; ++q) {
        const double z = (sS[q] - P.gc[(size_t)k * kMaxCV + q]) / P.gw[(size_t)k * kMaxCV + q];
        z2 += z * z;
      }
      const double e = P.gh[k] * exp(-0.5 * z2);
      V += e;
      for (int q = 0; q < nc; ++q) {
        const double w = P.gw[(size_t)k * kMaxCV + q];
        dV[q] -= e * (sS[q] - P.gc[(size_t)k * kMaxCV + q]) / (w * w);
      }
    }
  V = block_sum<kRedBlock>(V, sh);
#pragma unroll
  for (int q = 0; q < kMaxCV; ++q) dV[q] = block_sum<kRedBlock>(dV[q], sh);
  if (threadIdx.x == 0) {
    if (on && P.grad) {
      const int nl = P.N - 1;
      for (int q = 0; q < nc; ++q) {
        // ds/dx_k = +-(w_k / W) u for the atoms of group A / B (the same weights at both beads)
        const double *uN = sU[q][0], *u1 = sU[q][1];
        for (int k = P.cv_a[q]; k < P.cv_a[q + 1]; ++k) {
          const int a = P.gA[k];
          const double f = dV[q] * group_weight(sc, P.cv_com[q], a) / sW[q][0];
          for (int d = 0; d < 3; ++d) P.grad[3 * ((size_t)nl * P.Q + a) + d] += f * uN[d];
          if (P.cv_e2e[q])
            for (int d = 0; d < 3; ++d) P.grad[3 * (size_t)a + d] -= f * u1[d];
        }
        for (int k = P.cv_b[q]; k < P.cv_b[q + 1]; ++k) {
          const int b = P.gB[k];
          const double f = dV[q] * group_weight(sc, P.cv_com[q], b) / sW[q][1];
          for (int d = 0; d < 3; ++d) P.grad[3 * ((size_t)nl * P.Q + b) + d] -= f * uN[d];
          if (P.cv_e2e[q])
            for (int d = 0; d < 3; ++d) P.grad[3 * (size_t)b + d] += f * u1[d];
        }
      }
    }
    P.diag[2] = on ? V : 0.0;
    P.diag[3] = nc > 0 ? sS[0] : 0.0;
  }
}

// metadynamics deposition (one block per path): a Gaussian centred at the current CV values goes
// to row n_gauss of every path with CVs (the host counts the deposits); its width along CV q is
// the CV's own deposit width, or `width` where that is 0
__global__ void k_deposit(SysConsts sc, const PathDev* __restrict__ paths, double height, double width) {
  const PathDev& P = paths[blockIdx.x];
  if (threadIdx.x != 0 || P.n_cv < 1 || P.n_gauss >= kMaxGauss) return;
  for (int q = 0; q < P.n_cv; ++q) {
    double uN[3], u1[3], Wa, Wb;
    P.gc[(size_t)P.n_gauss * kMaxCV + q] = cv_value(sc, P, q, uN, u1, &Wa, &Wb);
    P.gw[(size_t)P.n_gauss * kMaxCV + q] = P.cv_width[q] > 0.0 ? P.cv_width[q] : width;
  }
  P.gh[P.n_gauss] = height;
}

// Ewald exclusion corrections: the reciprocal sum includes every excluded pair, so each gets
// phi_x(r) = -f q_i q_j erf(beta r) / r (no cutoff).  One thread per (excluded pair, bead):
// MODE 0 the force (and bead-1 energy partials), MODE 1 H eta, MODE 2 the FD difference of the
// force at R +- eps eta; +-f is added, fixed point, to the j-side sums of both atoms.
__device__ __forceinline__ void excl_terms(const SysConsts& sc, float r2, float qq, float* g, float* b, float* e) {
  const float rinv = rsqrtf(r2), r = r2 * rinv;
  const float er = erff(sc.ewb * r), c2e = sc.ewc2 * __expf(-sc.ewb2 * r2);
  // phi_x' = qq (erf / r^2 - c2E / r); g = -phi_x' / r; b = (phi_x'' + g) / r^2
  *g = -qq * rinv * rinv * (er * rinv - c2e);
  *b = -qq * rinv * rinv * rinv * (3.f * er * rinv * rinv - c2e * (3.f * rinv + 2.f * sc.ewb2 * r));
  *e = -qq * er * rinv;
}

// One thread per atom (caller order) and bead: the corrections of all its excluded pairs, summed
// in registers and added to the atom's own fixed-point j-side sums with a plain read-modify-write
// (the pair kernel has finished, and no other thread owns the row), so no atomics.  Each pair is
// evaluated from both ends; its energy is counted by the lower index.
template <int MODE>
__global__ void __launch_bounds__(kRedBlock) k_excl(SysConsts sc, const PathDev* __restrict__ paths, int n_begin) {
  __shared__ double sh[32];
  const int p = blockIdx.z, n = n_begin + blockIdx.y;
  const PathDev& P = paths[p];
  const int n_pass = MODE == 0 ? P.n_force : P.n_hvp;
  if (n >= n_pass) return;   // whole block
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  float en = 0.f;
  const int t0 = a < sc.Q ? sc.excl_off[a] : 0, t1 = a < sc.Q ? sc.excl_off[a + 1] : 0;
  if (t1 > t0) {
    const double qa = sc.qs[a];
    float ea[3] = {0.f, 0.f, 0.f};
    if (MODE >= 1) eta_of<float>(P, n, a, ea);
    float eps = 0.f;
    if (MODE == 2) {
      const float mx = __uint_as_float(P.etamax[n]);
      eps = (float)(mx > 0.f ? sc.fd_h / (double)mx : sc.fd_h);
    }
    float fa[3] = {0.f, 0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
      const int b = sc.excl_nb[t];
      float d[3];
      mi_diff<float>(sc, P, n, a, b, d);   // x_a - x_b
      const float qq = (float)(qa * sc.qs[b]);
      float f[3];
      if (MODE == 0) {
        float g, bb, e;
        excl_terms(sc, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], qq, &g, &bb, &e);
        for (int c = 0; c < 3; ++c) f[c] = g * d[c];
        if (a < b) en += e;
      } else {
        float eb[3], u[3];
        eta_of<float>(P, n, b, eb);
        for (int c = 0; c < 3; ++c) u[c] = ea[c] - eb[c];
        if (MODE == 1) {
          float g, bb, e;
          excl_terms(sc, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], qq, &g, &bb, &e);
          const float s = bb * (d[0] * u[0] + d[1] * u[1] + d[2] * u[2]);
          for (int c = 0; c < 3; ++c) f[c] = s * d[c] - g * u[c];   // A u
        } else {
          float fp[3], fm[3];
          for (int sg = 0; sg < 2; ++sg) {
            float w[3];
            for (int c = 0; c < 3; ++c) w[c] = d[c] + (sg ? -eps : eps) * u[c];
            float g, bb, e;
            excl_terms(sc, w[0] * w[0] + w[1] * w[1] + w[2] * w[2], qq, &g, &bb, &e);
            for (int c = 0; c < 3; ++c) (sg ? fm : fp)[c] = g * w[c];
          }
          for (int c = 0; c < 3; ++c) f[c] = -(fp[c] - fm[c]) / (2.f * eps);   // H eta = -dF/de
        }
      }
      for (int c = 0; c < 3; ++c) fa[c] += f[c];
    }
    unsigned long long* J = P.jacc + 3 * ((size_t)n * P.Qpad + P.slot[a]);
    for (int c = 0; c < 3; ++c) J[c] += (unsigned long long)__float2ll_rn(fa[c] * kFixScale);
  }
  if (MODE == 0 && n == 0) {
    const double tot = block_sum<kRedBlock>((double)en, sh);
    if (threadIdx.x == 0) P.e_excl[blockIdx.x] = tot;
  }
}

// fixed-order sums of the partial energies (10^4 - 10^5 per path) -> V_eff, one block per path
constexpr int kReduceBlock = 1024;
__global__ void __launch_bounds__(kReduceBlock)
    k_reduce(const PathDev* __restrict__ paths, int n_paths, const double* e_bond, int sb, int nb1,
                         const double* e_spring, int ss, int nb2, int n_excl_blk, double e_self, int n_pme_blk) {
  // e_bond: nb1 partials per path (stride sb); e_spring: nb2 partials per path (stride ss)
  __shared__ double sh[32];
  const int p = blockIdx.x;
  const PathDev& P = paths[p];
  double up = 0.0, ub = 0.0, es = 0.0;
  for (int k = threadIdx.x; k < P.meta[0]; k += blockDim.x) up += P.e_pair[k];
  if (P.e_excl)   // Ewald: exclusion corrections (self term added below)
    for (int k = threadIdx.x; k < n_excl_blk; k += blockDim.x) up += P.e_excl[k];
  if (P.pme_e)    // SPME reciprocal-space energy of bead 1
    for (int k = threadIdx.x; k < n_pme_blk; k += blockDim.x) up += P.pme_e[k];
  for (int k = threadIdx.x; k < nb1; k += blockDim.x) ub += e_bond[(size_t)p * sb + k];
  for (int k = threadIdx.x; k < nb2; k += blockDim.x) es += e_spring[(size_t)p * ss + k];
  up = block_sum<kReduceBlock>(up, sh);
  ub = block_sum<kReduceBlock>(ub, sh);
  es = block_sum<kReduceBlock>(es, sh);
  if (threadIdx.x == 0) {
    if (P.e_excl) up += e_self;
    const double U1 = up + ub;
    const double V = U1 + es + P.diag[2];
    P.diag[0] = U1;
    P.diag[1] = es;
    P.diag[4] = V;
    P.diag[5] = up;
    P.diag[6] = ub;
    if (P.veff_out) *P.veff_out = V;
  }
}

// ------------------------------------------------------------------------------------------
// integrator

// Philox-4x32-10 (Salmon et al., SC'11): four 32-bit words per (counter, key)
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__global__ void k_kick(int Q, const double* mass, double* vel, const double* grad, double half_dt) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;   // grid: (atoms, beads)
  if (a >= Q) return;
  const size_t t = 3 * ((size_t)blockIdx.y * Q + a);
  const double s = half_dt / mass[a];
  for (int d = 0; d < 3; ++d) vel[t + d] -= s * grad[t + d];
}

__global__ void k_drift(int Q, int N, const double* mass, double* x64, double* vel, float* x32, double dt, double c1,
                        double c2, double kT, uint64_t seed, const unsigned long long* step_ptr) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;   // grid: (atoms, beads)
  if (a >= Q) return;
  const unsigned long long step = *step_ptr;
  const int n = blockIdx.y;
  const size_t t = (size_t)n * Q + a;
  double* x = x64 + 3 * t;
  double* v = vel + 3 * t;
  for (int d = 0; d < 3; ++d) x[d] += 0.5 * dt * v[d];
  if (c2 > 0.0) {
    const uint4 w = philox(make_uint4((uint32_t)a, (uint32_t)n, (uint32_t)step, (uint32_t)(step >> 32)),
                           make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double inv32 = 2.3283064365386963e-10;   // 2^-32
    const double u1 = ((double)w.x + 1.0) * inv32, u2 = (double)w.y * inv32;
    const double u3 = ((double)w.z + 1.0) * inv32, u4 = (double)w.w * inv32;
    const double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
    double s1, c1p, s2, c2p;
    sincospi(2.0 * u2, &s1, &c1p);
    sincospi(2.0 * u4, &s2, &c2p);
    const double g[3] = {r1 * c1p, r1 * s1, r2 * c2p};
    const double sd = c2 * sqrt(kT / mass[a]);
    for (int d = 0; d < 3; ++d) v[d] = c1 * v[d] + sd * g[d];
  }
  for (int d = 0; d < 3; ++d) {
    x[d] += 0.5 * dt * v[d];
    x32[3 * t + d] = (float)x[d];
  }
}

__global__ void k_kinetic(int Q, int N, const double* mass, const double* vel, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int n = 0; n < N; ++n)
    for (int a = threadIdx.x; a < Q; a += blockDim.x) {
      const double* v = vel + 3 * ((size_t)n * Q + a);
      s += 0.5 * mass[a] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
  s = block_sum<kRedBlock>(s, sh);
  if (threadIdx.x == 0) *out = s;
}

inline int nblk(long long n, int bs) { return (int)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_e1(const SysConsts& sc, const PathDev* d_paths, int n_paths, int max_qpad, int max_beads, Launch L,
                      double* e_bond, int nbx) {
  dim3 grid(nbx, max_beads, n_paths);
  if (sc.precision == 1) k_e1<double><<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_paths, e_bond, nbx);
  else k_e1_mixed<<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_paths, e_bond, nbx);
  (void)max_qpad;
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_e2(const SysConsts& sc, const PathDev* d_paths, int n_paths, int max_qpad, int max_beads, Launch L,
                      double* e_spring, int nbx, int n_begin, int n_count) {
  if (n_count < 0) n_count = max_beads;
  if (n_count == 0) return cudaSuccess;
  dim3 grid(nbx, n_count, n_paths);
  const bool fd = sc.hvp_mode == 1;
  (void)max_qpad;
  if (sc.precision == 1) {
    if (fd) k_e2<double, true><<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_paths, e_spring, nbx, max_beads, n_begin);
    else k_e2<double, false><<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_paths, e_spring, nbx, max_beads, n_begin);
  } else {
    if (fd) k_e2_mixed<true><<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_paths, e_spring, nbx, max_beads, n_begin);
    else k_e2_mixed<false><<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_paths, e_spring, nbx, max_beads, n_begin);
  }
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_excl(const SysConsts& sc, const PathDev* d_paths, int n_paths, int max_beads, int mode, Launch L,
                        int n_begin, int n_count) {
  if (sc.elec != 1 || sc.n_excl == 0) return cudaSuccess;
  if (n_count < 0) n_count = max_beads;
  if (n_count == 0) return cudaSuccess;
  const dim3 grid((sc.Q + kRedBlock - 1) / kRedBlock, n_count, n_paths);
  if (mode == 0) k_excl<0><<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_begin);
  else if (mode == 1) k_excl<1><<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_begin);
  else k_excl<2><<<grid, kRedBlock, 0, L.st>>>(sc, d_paths, n_begin);
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_deposit(const SysConsts& sc, const PathDev* d_paths, int n_paths, double height, double width,
                           Launch L) {
  k_deposit<<<n_paths, 32, 0, L.st>>>(sc, d_paths, height, width);
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_bias(const SysConsts& sc, const PathDev* d_paths, int n_paths, Launch L) {
  k_bias<<<n_paths, kRedBlock, 0, L.st>>>(sc, d_paths, n_paths);
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_reduce(const SysConsts& sc, const PathDev* d_paths, int n_paths, Launch L, const double* e_bond,
                          int sb, int nb1, const double* e_spring, int ss, int nb2) {
  k_reduce<<<n_paths, kReduceBlock, 0, L.st>>>(d_paths, n_paths, e_bond, sb, nb1, e_spring, ss, nb2,
                                             excl_energy_blocks(sc), sc.e_self,
                                             pme_energy_blocks(sc));
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_kick(const SysConsts& sc, double* vel, const double* grad, int N, double half_dt, Launch L) {
  k_kick<<<dim3(nblk(sc.Q, kRedBlock), N), kRedBlock, 0, L.st>>>(sc.Q, sc.mass, vel, grad, half_dt);
  ++*L.counter;
  return cudaGetLastError();
}

__global__ void k_step_inc(unsigned long long* step) { *step += 1ull; }

cudaError_t launch_step_inc(unsigned long long* step, Launch L) {
  k_step_inc<<<1, 1, 0, L.st>>>(step);
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_drift(const SysConsts& sc, double* x64, double* vel, float* x32, int N, double dt, double gamma,
                         double kT, uint64_t seed, const unsigned long long* step, Launch L) {
  const double c1 = gamma > 0.0 ? exp(-gamma * dt) : 1.0;
  const double c2 = gamma > 0.0 ? sqrt(1.0 - c1 * c1) : 0.0;
  k_drift<<<dim3(nblk(sc.Q, kRedBlock), N), kRedBlock, 0, L.st>>>(sc.Q, N, sc.mass, x64, vel, x32, dt, c1, c2, kT,
                                                                  seed, step);
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t launch_kinetic(const SysConsts& sc, const double* vel, int N, double* out, Launch L) {
  k_kinetic<<<1, kRedBlock, 0, L.st>>>(sc.Q, N, sc.mass, vel, out);
  ++*L.counter;
  return cudaGetLastError();
}

}  // namespace mop
