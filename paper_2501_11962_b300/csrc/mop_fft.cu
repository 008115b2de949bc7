// Batched 3-D FFTs of the SPME grids: the forward real-to-complex transform of every bead's charge
// grid, the multiplication by the Ewald reciprocal kernel theta, and the inverse complex-to-real
// transform back to the potential grid, in five passes over the half spectrum:
//   z-lines  R2C   the int64 fixed-point charges converted on load, two real lines per complex
//                  transform (packed as real and imaginary parts, separated afterwards)
//   y-lines  C2C   forward
//   x-lines  C2C   forward, times theta (with the bead-1 energy 1/2 sum theta |F|^2), inverse
//   y-lines  C2C   inverse
//   z-lines  C2R   two real lines per complex transform
// Every line is transformed in shared memory by a self-sorting (Stockham) mixed-radix FFT: with
// L the length of the sub-transforms done so far and M' = N / (L r), a radix-r stage maps
//   A'[j + L t + L r m'] = sum_s W_r^{s t} W_N^{s j M'} A[j + L (m' + M' s)]
// (j < L, t < r, m' < M'), starting from A = x (L = 1) and ending with the sorted DFT (L = N).
// Radices 8, 4, 2, 3, 5, 7; the inverse uses conjugate twiddles and is not normalised.
#include <cmath>
#include <vector>

#include "mop_host.h"

namespace mop {
namespace {

// W_r^k = (cos 2 pi k / r, sin 2 pi k / r) for the odd radices (the forward DFT conjugates them)
__constant__ float kC3[3] = {1.000000000e+00f, -5.000000000e-01f, -5.000000000e-01f};
__constant__ float kS3[3] = {0.000000000e+00f, 8.660254038e-01f, -8.660254038e-01f};
__constant__ float kC5[5] = {1.000000000e+00f, 3.090169944e-01f, -8.090169944e-01f, -8.090169944e-01f,
                             3.090169944e-01f};
__constant__ float kS5[5] = {0.000000000e+00f, 9.510565163e-01f, 5.877852523e-01f, -5.877852523e-01f,
                             -9.510565163e-01f};
__constant__ float kC7[7] = {1.000000000e+00f, 6.234898019e-01f, -2.225209340e-01f, -9.009688679e-01f,
                             -9.009688679e-01f, -2.225209340e-01f, 6.234898019e-01f};
__constant__ float kS7[7] = {0.000000000e+00f, 7.818314825e-01f, 9.749279122e-01f, 4.338837391e-01f,
                             -4.338837391e-01f, -9.749279122e-01f, -7.818314825e-01f};

// lines a block transforms together, one per lane (16-line tiles, two butterflies per warp,
// measured slower: 310 against 286 us per convolution of 15 beads of a 96^3 grid)
constexpr int kFftLanes = 32;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// v_t = sum_s u_s W_R^{-sign s t}: sign = +1 forward (W = exp(-2 pi i / R)), -1 inverse
template <int R>
__device__ __forceinline__ void small_dft(const float2 (&u)[R], float2 (&v)[R], float sign) {
  if constexpr (R == 2) {
    v[0] = cadd(u[0], u[1]);
    v[1] = csub(u[0], u[1]);
  } else if constexpr (R == 8) {
    // two radix-4 DFTs of the even and odd inputs, combined with W_8^t (c = sqrt(2) / 2)
    const float c = 7.071067812e-01f;
    float2 e4[4], o4[4], ev[4], ov[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      e4[k] = u[2 * k];
      o4[k] = u[2 * k + 1];
    }
    small_dft<4>(e4, ev, sign);
    small_dft<4>(o4, ov, sign);
    // W_8^t o for t = 1, 2, 3 (forward: W_8 = c (1 - i); inverse: conjugate)
    const float2 o1 = make_float2(c * (ov[1].x + sign * ov[1].y), c * (ov[1].y - sign * ov[1].x));
    const float2 o2 = make_float2(sign * ov[2].y, -sign * ov[2].x);
    const float2 o3 = make_float2(c * (-ov[3].x + sign * ov[3].y), c * (-ov[3].y - sign * ov[3].x));
    v[0] = cadd(ev[0], ov[0]);
    v[4] = csub(ev[0], ov[0]);
    v[1] = cadd(ev[1], o1);
    v[5] = csub(ev[1], o1);
    v[2] = cadd(ev[2], o2);
    v[6] = csub(ev[2], o2);
    v[3] = cadd(ev[3], o3);
    v[7] = csub(ev[3], o3);
  } else if constexpr (R == 4) {
    // multiplication by -i (forward) or +i (inverse): (x, y) -> (sign y, -sign x)
    const float2 a = cadd(u[0], u[2]), b = csub(u[0], u[2]), c = cadd(u[1], u[3]), d = csub(u[1], u[3]);
    const float2 dr = make_float2(sign * d.y, -sign * d.x);
    v[0] = cadd(a, c);
    v[1] = cadd(b, dr);
    v[2] = csub(a, c);
    v[3] = csub(b, dr);
  } else {
    const float* C = R == 3 ? kC3 : (R == 5 ? kC5 : kC7);
    const float* S = R == 3 ? kS3 : (R == 5 ? kS5 : kS7);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float2 acc = u[0];
#pragma unroll
      for (int s = 1; s < R; ++s) {
        const int k = (s * t) % R;
        const float2 w = make_float2(C[k], -sign * S[k]);
        acc = cadd(acc, cmul(u[s], w));
      }
      v[t] = acc;
    }
  }
}

// One radix-R stage of the Stockham transform of up to 32 lines of length N held element-major:
// element k of line l at k * LS + l in both buffers (LS = lines + 1, so that the rows of a
// column fall in different banks).  Lane l of every warp works on line l; the warps share out
// the butterflies b = (j, m') of the stage, whose twiddles are the same for the whole warp;
// tw[i] = exp(-2 pi i i / N).
template <int R>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ in, float2* __restrict__ out, int N, int LS,
                                          int nl, int L, const float2* __restrict__ tw, float sign) {
  const int Lp = L * R, Mp = N / Lp, nb = N / R;
  // kFftLanes lanes per line group: a warp runs 32 / kFftLanes butterflies at once
  const int l = threadIdx.x % kFftLanes, w0 = threadIdx.x / kFftLanes, nw = blockDim.x / kFftLanes;
  if (l >= nl) return;
  for (int b = w0; b < nb; b += nw) {
    const int mp = b / L, j = b - mp * L;
    float2 wt[R];
#pragma unroll
    for (int s = 1; s < R; ++s) {
      wt[s] = __ldg(&tw[s * j * Mp]);   // s j M' < N
      wt[s].y *= sign;
    }
    const float2* x = in + (j + L * mp) * LS + l;
    float2 u[R], v[R];
    u[0] = x[0];
#pragma unroll
    for (int s = 1; s < R; ++s) u[s] = cmul(x[L * Mp * s * LS], wt[s]);
    small_dft<R>(u, v, sign);
    float2* y = out + (j + Lp * mp) * LS + l;
#pragma unroll
    for (int q = 0; q < R; ++q) y[L * q * LS] = v[q];
  }
}

// All stages; returns the buffer (a or b) that holds the result.  Every thread of the block must
// call it.
__device__ __forceinline__ float2* fft_lines(float2* a, float2* b, const FftAxis& ax, int LS, int nl, bool inverse) {
  const float sign = inverse ? -1.f : 1.f;
  int L = 1;
  float2* in = a;
  float2* out = b;
  for (int st = 0; st < ax.nr; ++st) {
    const int r = ax.radix[st];
    __syncthreads();
    switch (r) {
      case 8: fft_stage<8>(in, out, ax.n, LS, nl, L, ax.tw, sign); break;
      case 4: fft_stage<4>(in, out, ax.n, LS, nl, L, ax.tw, sign); break;
      case 2: fft_stage<2>(in, out, ax.n, LS, nl, L, ax.tw, sign); break;
      case 3: fft_stage<3>(in, out, ax.n, LS, nl, L, ax.tw, sign); break;
      case 5: fft_stage<5>(in, out, ax.n, LS, nl, L, ax.tw, sign); break;
      default: fft_stage<7>(in, out, ax.n, LS, nl, L, ax.tw, sign); break;
    }
    L *= r;
    float2* tmp = in;
    in = out;
    out = tmp;
  }
  __syncthreads();
  return in;
}

constexpr int kFftThreads = 256;
constexpr float kGridInvF = 1.0f / 1099511627776.0f;   // 2^-40: unit of the fixed-point charge grids

// z-lines, forward: real lines r0 = 2p, r1 = 2p + 1 of length N (int64 fixed point, converted
// here) as one complex line z = a + i b; after the transform A[k] = (Z[k] + conj Z[N-k]) / 2 and
// B[k] = (Z[k] - conj Z[N-k]) / (2 i), k < N / 2 + 1, go to the half spectra of lines r0 and r1.
// Flat element idx of the block's range belongs to pair idx / N (multiply-high division).
__global__ void __launch_bounds__(kFftThreads) k_fft_z_r2c(const unsigned long long* __restrict__ q,
                                                           float2* __restrict__ c, long long n_lines, int kc,
                                                           unsigned mkc, FftAxis ax, int pairs_per_block) {
  extern __shared__ float2 sm[];
  const int N = ax.n, LS = pairs_per_block + 1;
  float2* a = sm;
  float2* b = sm + N * LS;
  const long long p0 = (long long)blockIdx.x * pairs_per_block;
  const long long n_pairs = (n_lines + 1) / 2;
  const int np = (int)min((long long)pairs_per_block, n_pairs - p0);
  const unsigned long long* q0 = q + 2 * p0 * N;
  const bool odd_tail = 2 * (p0 + np) > n_lines;   // the last pair has no second line
  for (int idx = threadIdx.x; idx < np * N; idx += blockDim.x) {
    const int l = (int)__umulhi((unsigned)idx, ax.magic), k = idx - l * N;
    const float re = (float)(long long)q0[(2 * l) * N + k] * kGridInvF;
    const float im = (odd_tail && l == np - 1) ? 0.f : (float)(long long)q0[(2 * l + 1) * N + k] * kGridInvF;
    a[k * LS + l] = make_float2(re, im);
  }
  const float2* z = fft_lines(a, b, ax, LS, np, false);
  float2* c0 = c + 2 * p0 * kc;
  for (int idx = threadIdx.x; idx < np * kc; idx += blockDim.x) {
    const int l = (int)__umulhi((unsigned)idx, mkc), k = idx - l * kc;
    const float2 x = z[k * LS + l], y = z[(k == 0 ? 0 : N - k) * LS + l];   // Z[k], Z[N - k]
    c0[(2 * l) * kc + k] = make_float2(0.5f * (x.x + y.x), 0.5f * (x.y - y.y));
    if (!(odd_tail && l == np - 1)) c0[(2 * l + 1) * kc + k] = make_float2(0.5f * (x.y + y.y), -0.5f * (x.x - y.x));
  }
}

// z-lines, inverse: half spectra A (line 2p) and B (line 2p + 1), extended by Hermitian symmetry
// (the imaginary parts at k = 0 and k = N / 2 dropped, as for any real inverse), combined as
// Z = A + i B and transformed back: the real part is line 2p, the imaginary part line 2p + 1.
__global__ void __launch_bounds__(kFftThreads) k_fft_z_c2r(const float2* __restrict__ c, float* __restrict__ out,
                                                           long long n_lines, int kc, FftAxis ax,
                                                           int pairs_per_block) {
  extern __shared__ float2 sm[];
  const int N = ax.n, LS = pairs_per_block + 1;
  float2* a = sm;
  float2* b = sm + N * LS;
  const long long p0 = (long long)blockIdx.x * pairs_per_block;
  const long long n_pairs = (n_lines + 1) / 2;
  const int np = (int)min((long long)pairs_per_block, n_pairs - p0);
  const bool odd_tail = 2 * (p0 + np) > n_lines;
  const float2* c0 = c + 2 * p0 * kc;
  for (int idx = threadIdx.x; idx < np * N; idx += blockDim.x) {
    const int l = (int)__umulhi((unsigned)idx, ax.magic), k = idx - l * N;
    const bool mirror = k >= kc;
    const int kk = mirror ? N - k : k;
    float2 A = c0[(2 * l) * kc + kk];
    float2 B = (odd_tail && l == np - 1) ? make_float2(0.f, 0.f) : c0[(2 * l + 1) * kc + kk];
    if (kk == 0 || 2 * kk == N) {
      A.y = 0.f;
      B.y = 0.f;
    }
    if (mirror) {
      A.y = -A.y;
      B.y = -B.y;
    }
    a[k * LS + l] = make_float2(A.x - B.y, A.y + B.x);
  }
  const float2* z = fft_lines(a, b, ax, LS, np, true);
  float* o0 = out + 2 * p0 * N;
  for (int idx = threadIdx.x; idx < np * N; idx += blockDim.x) {
    const int l = (int)__umulhi((unsigned)idx, ax.magic), k = idx - l * N;
    const float2 v = z[k * LS + l];
    o0[(2 * l) * N + k] = v.x;
    if (!(odd_tail && l == np - 1)) o0[(2 * l + 1) * N + k] = v.y;
  }
}

// Strided lines of the half spectrum: plane blockIdx.y starts at plane * plane_stride; its lines
// are the cw contiguous columns, element k of column col at k * es + col.  A block takes up to 32
// consecutive columns: lane = column, warp = row, the same element-major layout as in shared
// memory (coalesced, no transposition, no division).
// KIND 0: forward; 1: inverse; 2: forward, times theta[k * cw + col], inverse, and with `energy`
// the block's part of 1/2 sum theta |F|^2 (weight 2 off the kz = 0 and Nyquist planes) of plane 0.
template <int KIND>
__global__ void __launch_bounds__(kFftThreads) k_fft_strided(float2* __restrict__ c, long long plane_stride,
                                                             int es, int cw, FftAxis ax, int lines_per_block,
                                                             const float* __restrict__ theta, int kc, int k3,
                                                             double* energy) {
  extern __shared__ float2 sm[];
  __shared__ double red[kFftThreads / 32];
  const int N = ax.n, LS = lines_per_block + 1;
  float2* a = sm;
  float2* b = sm + N * LS;
  const int col0 = blockIdx.x * lines_per_block;
  const int nl = min(lines_per_block, cw - col0);
  float2* base = c + (long long)blockIdx.y * plane_stride + col0;
  const int tx = threadIdx.x % kFftLanes, ty = threadIdx.x / kFftLanes, nrow = blockDim.x / kFftLanes;
  if (tx < nl)
    for (int k = ty; k < N; k += nrow) a[k * LS + tx] = base[(long long)k * es + tx];
  float2* z = fft_lines(a, b, ax, LS, nl, KIND == 1);
  if constexpr (KIND == 2) {
    double e = 0.0;
    const bool want = energy && blockIdx.y == 0;
    if (tx < nl) {
      const int kz = (col0 + tx) % kc;
      const double wz = (kz == 0 || 2 * kz == k3) ? 0.5 : 1.0;
      for (int k = ty; k < N; k += nrow) {
        const float th = __ldg(&theta[(long long)k * cw + col0 + tx]);
        float2 v = z[k * LS + tx];
        if (want) e += wz * (double)th * ((double)v.x * v.x + (double)v.y * v.y);
        v.x *= th;
        v.y *= th;
        z[k * LS + tx] = v;
      }
    }
    if (want) {
      e = warp_sum(e);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    }
    float2* other = z == a ? b : a;
    z = fft_lines(z, other, ax, LS, nl, true);
    if (want && threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kFftThreads / 32; ++w) t += red[w];
      energy[blockIdx.x] = t;
    }
  }
  if (tx < nl)
    for (int k = ty; k < N; k += nrow) base[(long long)k * es + tx] = z[k * LS + tx];
}

}  // namespace

bool fft_factor(int n, int* radix, int* nr) {
  *nr = 0;
  for (int r : {8, 4, 2, 3, 5, 7})
    while (n % r == 0 && *nr < kFftMaxStages) {
      radix[(*nr)++] = r;
      n /= r;
    }
  return n == 1;
}

cudaError_t fft_axis_make(int n, DevBuf<float2>& tw, FftAxis* ax) {
  ax->n = n;
  // idx / n = umulhi(idx, magic) exactly while idx n < 2^32 (idx < 2^21 here)
  ax->magic = n > 0 ? (unsigned)(((1ull << 32) + (unsigned long long)n - 1) / (unsigned long long)n) : 0u;
  if (n < 2 || n > kFftMaxLen || !fft_factor(n, ax->radix, &ax->nr)) return cudaErrorInvalidValue;
  std::vector<float2> h(n);
  for (int i = 0; i < n; ++i) {
    const double t = 2.0 * M_PI * (double)i / (double)n;
    h[i] = make_float2((float)std::cos(t), (float)-std::sin(t));
  }
  cudaError_t e = tw.ensure(n);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(tw.p, h.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
  ax->tw = tw.p;
  return e;
}

// dynamic shared memory of a pass over lines of length n, `lines` at a time (two buffers)
inline size_t fft_smem(int n, int lines) { return 2 * sizeof(float2) * (size_t)n * (size_t)(lines + 1); }

template <class K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_fft_convolve(const SysConsts& sc, const FftAxis* ax, const unsigned long long* q, float2* c,
                                float* out, int beads, double* energy, Launch L) {
  const int K1 = sc.pme_K[0], K2 = sc.pme_K[1], K3 = sc.pme_K[2], kc = sc.pme_kc3;
  const long long nz = (long long)beads * K1 * K2;   // z-lines
  const int ppb = fft_lines_per_block(K3, 1 << 30);
  const unsigned zblocks = (unsigned)(((nz + 1) / 2 + ppb - 1) / ppb);
  const size_t zsm = fft_smem(K3, ppb);
  const unsigned mkc = (unsigned)(((1ull << 32) + (unsigned long long)kc - 1) / (unsigned long long)kc);
  cudaError_t e;
  if ((e = allow_smem(k_fft_z_r2c, zsm)) != cudaSuccess || (e = allow_smem(k_fft_z_c2r, zsm)) != cudaSuccess)
    return e;
  k_fft_z_r2c<<<zblocks, kFftThreads, zsm, L.st>>>(q, c, nz, kc, mkc, ax[2], ppb);
  // y-lines: planes (bead, x), columns kz, elements y at stride kc
  const int ycw = kc, ylpb = fft_lines_per_block(K2, ycw);
  const dim3 ygrid((unsigned)((ycw + ylpb - 1) / ylpb), (unsigned)(beads * K1));
  const size_t ysm = fft_smem(K2, ylpb);
  // x-lines: planes (bead), columns (y, kz), elements x at stride K2 kc
  const int xcw = K2 * kc, xlpb = fft_lines_per_block(K1, xcw);
  const dim3 xgrid((unsigned)((xcw + xlpb - 1) / xlpb), (unsigned)beads);
  const size_t xsm = fft_smem(K1, xlpb);
  if ((e = allow_smem(k_fft_strided<0>, ysm)) != cudaSuccess || (e = allow_smem(k_fft_strided<1>, ysm)) != cudaSuccess ||
      (e = allow_smem(k_fft_strided<2>, xsm)) != cudaSuccess)
    return e;
  k_fft_strided<0><<<ygrid, kFftThreads, ysm, L.st>>>(c, (long long)K2 * kc, kc, ycw, ax[1], ylpb, nullptr, kc, K3,
                                                      nullptr);
  k_fft_strided<2><<<xgrid, kFftThreads, xsm, L.st>>>(c, (long long)K1 * K2 * kc, K2 * kc, xcw, ax[0], xlpb,
                                                      sc.pme_theta, kc, K3, energy);
  k_fft_strided<1><<<ygrid, kFftThreads, ysm, L.st>>>(c, (long long)K2 * kc, kc, ycw, ax[1], ylpb, nullptr, kc, K3,
                                                      nullptr);
  k_fft_z_c2r<<<zblocks, kFftThreads, zsm, L.st>>>(c, out, nz, kc, ax[2], ppb);
  *L.counter += 5;
  return cudaGetLastError();
}

}  // namespace mop
