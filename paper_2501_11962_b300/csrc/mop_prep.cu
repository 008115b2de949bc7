// Spatial sort, clusters and the cluster-pair list of one path.
//
// The paper evaluates each bead's forces with GROMACS' own neighbour search (Sec. 2.1, one
// bead per processing element).  Here all beads of a path share ONE sort and ONE cluster-pair
// list: atoms are ordered by the reference bead (bead 1) into x-y columns and z, cut into
// clusters of 8, and every cluster gets the union of its bounding boxes over all beads (each
// bead's atom taken at the periodic image nearest its reference position).  A cluster pair is
// listed (with its periodic image) when the union boxes are closer than rc, so the list is
// exact for every bead without a Verlet buffer.  Coordinates are stored relative to the
// cluster centre so that FP32 pair differences stay accurate in large boxes.
#include <algorithm>
#include <cstdio>

#include "mop_host.h"

namespace mop {
namespace {

__device__ __forceinline__ double coord(const float* x32, const double* x64, size_t k) {
  return x64 ? x64[k] : (double)x32[k];
}

// exclusive scan of one value per thread over a 1024-thread block; *total gets the block sum
__device__ int block_excl_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const int pre = (w > 0 ? sh[w - 1] : 0) + x - v;
  *total = sh[nw - 1];
  __syncthreads();
  return pre;
}

// reference wrap of bead 1, column index and column counts
__global__ void k_ref_columns(SysConsts sc, const float* x32, const double* x64, int ncx, int ncy, double wx,
                              double wy, double* ref, float* reff, int* colid, int* colcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.Q) return;
  double r[3];
  for (int d = 0; d < 3; ++d) {
    const double v = coord(x32, x64, 3 * (size_t)i + d);
    double w = v - sc.L[d] * floor(v * sc.invL[d]);
    if (w >= sc.L[d]) w -= sc.L[d];
    if (w < 0.0) w = 0.0;
    r[d] = w;
    ref[3 * i + d] = w;
    if (reff) reff[3 * i + d] = (float)w;
  }
  // fmax/fmin also map a NaN coordinate to a valid column (the result is then rejected later)
  const int cx = (int)fmin(fmax(r[0] / wx, 0.0), (double)(ncx - 1));
  const int cy = (int)fmin(fmax(r[1] / wy, 0.0), (double)(ncy - 1));
  const int col = cx * ncy + cy;
  colid[i] = col;
  atomicAdd(&colcnt[col], 1);
}

// colinfo[3c] = first atom of column c in colatoms, [3c+1] = first slot (padded to 8),
// [3c+2] = fill cursor; meta[0] = number of clusters
__global__ void k_scan_columns(const int* colcnt, int ncol, int* colinfo, int* meta) {
  __shared__ int sh[32];
  int carry = 0, pcarry = 0;
  for (int base = 0; base < ncol; base += blockDim.x) {
    const int c = base + threadIdx.x;
    const int cnt = c < ncol ? colcnt[c] : 0;
    const int pad = (cnt + kCL - 1) / kCL * kCL;
    int tot, ptot;
    const int pre = block_excl_scan(cnt, sh, &tot);
    const int ppre = block_excl_scan(pad, sh, &ptot);
    if (c < ncol) {
      colinfo[3 * c] = carry + pre;
      colinfo[3 * c + 1] = pcarry + ppre;
      colinfo[3 * c + 2] = carry + pre;
    }
    carry += tot;
    pcarry += ptot;
  }
  if (threadIdx.x == 0) meta[0] = pcarry / kCL;
}

__global__ void k_fill_columns(int Q, const int* colid, int* colinfo, int* colatoms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q) return;
  const int pos = atomicAdd(&colinfo[3 * colid[i] + 2], 1);
  colatoms[pos] = i;
}

// rank inside the column by (z, atom index): deterministic slot of every atom.  One block per
// column; the column's (z, index) pairs pass through shared memory in tiles, and each thread
// counts the atoms that precede its own.  The wrapped z is >= 0 (or NaN, rejected later), so
// its bit pattern, with -0 taken as +0, orders like the value: integer compares instead of the
// FP64 pipe.
constexpr int kRankTile = 1024;
__device__ __forceinline__ unsigned long long z_key(double z) {
  return z == 0.0 ? 0ull : (unsigned long long)__double_as_longlong(z);
}
__global__ void k_rank(const double* ref, const int* colcnt, const int* colinfo, const int* colatoms, int* perm,
                       int* slot) {
  __shared__ unsigned long long zs[kRankTile];
  __shared__ int js[kRankTile];
  const int col = blockIdx.x;
  const int st = colinfo[3 * col], cnt = colcnt[col], s0 = colinfo[3 * col + 1];
  for (int base = 0; base < cnt; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const int i = k < cnt ? colatoms[st + k] : -1;
    const unsigned long long zi = i >= 0 ? z_key(ref[3 * i + 2]) : 0ull;
    int rank = 0;
    for (int t0 = 0; t0 < cnt; t0 += kRankTile) {
      const int nt = min(kRankTile, cnt - t0);
      __syncthreads();
      for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const int j = colatoms[st + t0 + t];
        js[t] = j;
        zs[t] = z_key(ref[3 * j + 2]);
      }
      __syncthreads();
      if (i >= 0)
        for (int t = 0; t < nt; ++t) rank += (zs[t] < zi) || (zs[t] == zi && js[t] < i);
    }
    if (i >= 0) {
      perm[s0 + rank] = i;
      slot[i] = s0 + rank;
    }
  }
}

// Mixed precision: the caller's FP32 coordinate x taken at the periodic image nearest its
// reference r, x - k L, as an exact double-float (FP32 pipes only; k L with L = (Lf, Llo) and
// k Lf formed exactly by an FMA).  Every FP32-path kernel picks k by the same FP32 formula.
__device__ __forceinline__ df aligned_df(const SysConsts& sc, float x, float r, int d) {
  const float k = rintf((x - r) * sc.invLf[d]);
  const float p = k * sc.Lf[d];
  const float pe = fmaf(k, sc.Lf[d], -p);
  const df t = two_sum(x, -p);
  return fast_two_sum(t.hi, (t.lo - pe) - k * sc.Llo[d]);
}

// union bounding box of each cluster over all beads (mixed precision); one warp per cluster,
// lanes over beads.  Coordinates are rounded to FP32 after alignment, so the half extents get
// a slack of a few units in the last place of the box size.
__global__ void k_cluster_bbox32(SysConsts sc, const float* x32, int N, const float* reff, const int* perm,
                                 const int* meta, int max_clu, double margin, double* center, float* hext, int* molr,
                                 unsigned* emax) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= max_clu || c >= meta[0]) return;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int atoms[kCL];
#pragma unroll
  for (int k = 0; k < kCL; ++k) atoms[k] = perm[c * kCL + k];
  const size_t Q3 = 3 * (size_t)sc.Q;
  for (int b = lane; b < N; b += 32) {
#pragma unroll
    for (int k = 0; k < kCL; ++k) {
      const int a = atoms[k];
      if (a < 0) continue;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const df v = aligned_df(sc, x32[b * Q3 + 3 * (size_t)a + d], reff[3 * a + d], d);
        const float f = v.hi + v.lo;
        lo[d] = fminf(lo[d], f);
        hi[d] = fmaxf(hi[d], f);
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  }
  if (lane == 0) {
    int m0 = 0x7fffffff, m1 = -0x7fffffff;
    for (int k = 0; k < kCL; ++k)
      if (atoms[k] >= 0) {
        m0 = min(m0, sc.mol[atoms[k]]);
        m1 = max(m1, sc.mol[atoms[k]]);
      }
    molr[2 * c] = m0;
    molr[2 * c + 1] = m1;
    for (int d = 0; d < 3; ++d) {
      const float cen = 0.5f * (lo[d] + hi[d]);
      const float ext = fmaxf(hi[d] - cen, cen - lo[d]);
      // |coordinate| < 2^k: the FP32 roundings above stay below 4 ulps of that size
      const float e = ext + (fabsf(cen) + ext) * 4.8e-7f + (float)margin + 1e-6f;
      center[3 * c + d] = widen(cen);
      hext[3 * c + d] = e;
      atomicMax(&emax[d], __float_as_uint(e));
    }
  }
}

// Mixed precision: cluster-local coordinates x - C of every bead (xq, with q sqrt(f) in w) and
// each atom's union sphere over the beads (abox), one thread per slot looping over the beads.
// Padding slots get far-away dummy coordinates, zero eta and an empty sphere.
__global__ void k_local_box32(SysConsts sc, const float* x32, int N, const float* reff, const int* perm,
                              const int* meta, int max_slots, const double* center, double margin, float4* xq, int* ts,
                              float4* eta32, float4* abox) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= meta[0] * kCL) return;
  const int a = perm[s];
  if (a < 0) {
    const float dmy = kDummyCoord + 3.0f * (float)(s & (kCL - 1));
    for (int b = 0; b < N; ++b) {
      const size_t o = (size_t)b * max_slots + s;
      xq[o] = make_float4(dmy, dmy, dmy, 0.0f);
      eta32[o] = make_float4(0.f, 0.f, 0.f, 0.f);   // read as j-atoms by the HVP kernels
    }
    ts[s] = 0;
    abox[s] = make_float4(kDummyCoord, kDummyCoord, kDummyCoord, -1.0f);
    return;
  }
  const int c = s / kCL;
  float cen[3], r[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    cen[d] = (float)center[3 * c + d];   // exactly representable
    r[d] = reff[3 * a + d];
  }
  const float q = (float)sc.qs[a];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  const size_t Q3 = 3 * (size_t)sc.Q;
#pragma unroll 4
  for (int b = 0; b < N; ++b) {
    float v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const df A = aligned_df(sc, x32[b * Q3 + 3 * (size_t)a + d], r[d], d);
      const df t = two_sum(A.hi, -cen[d]);
      v[d] = t.hi + (t.lo + A.lo);
      lo[d] = fminf(lo[d], v[d]);
      hi[d] = fmaxf(hi[d], v[d]);
    }
    xq[(size_t)b * max_slots + s] = make_float4(v[0], v[1], v[2], q);
  }
  ts[s] = sc.type[a];
  float cf[3], h2 = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    cf[d] = 0.5f * (lo[d] + hi[d]);
    const float h = fmaxf(hi[d] - cf[d], cf[d] - lo[d]);
    h2 = fmaf(h, h, h2);
  }
  // local coordinates are below a few nm: 1e-6 nm covers every FP32 rounding here
  abox[s] = make_float4(cf[0], cf[1], cf[2], sqrtf(h2) * 1.000001f + (float)margin + 1e-6f);
}

// Mixed precision, reaction field, bead-lane pair kernels: the same cluster-local coordinates and
// atom spheres as k_local_box32, written directly in the bead-lane layout the pair kernels read,
// xb [group][slot][3][32] float2 (lane l holds beads 64 g + l and 64 g + 32 + l; beads past
// n_rows repeat the last row, as the transposition does), and in xq for bead 1 only (its row
// carries the charges and the bead-1 energy's coordinates).  One warp per slot, lanes over
// beads, so that the stores of xb are whole 256-byte rows.  The sphere's bounds are warp minima
// and maxima, which do not depend on the order, so abox has the bits of k_local_box32's.
__global__ void __launch_bounds__(256) k_local_box32_bl(SysConsts sc, const float* x32, int N, int n_rows,
                                                        const float* reff, const int* perm, const int* meta,
                                                        int max_slots, const double* center, double margin,
                                                        float4* xq, float2* xb, int* ts, float4* eta32, float4* abox) {
  const int lane = threadIdx.x & 31;
  const int s = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (s >= max_slots || s >= meta[0] * kCL) return;   // warp-uniform
  const int a = perm[s];
  const int groups = (n_rows + kBLBeads - 1) / kBLBeads;
  if (a < 0) {
    const float dmy = kDummyCoord + 3.0f * (float)(s & (kCL - 1));
    for (int g = 0; g < groups; ++g) {
      float2* o = xb + ((size_t)g * max_slots + s) * 3 * 32 + lane;
#pragma unroll
      for (int c = 0; c < 3; ++c) o[c * 32] = make_float2(dmy, dmy);
    }
    for (int b = lane; b < N; b += 32) eta32[(size_t)b * max_slots + s] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane == 0) {
      xq[s] = make_float4(dmy, dmy, dmy, 0.0f);
      ts[s] = 0;
      abox[s] = make_float4(kDummyCoord, kDummyCoord, kDummyCoord, -1.0f);
    }
    return;
  }
  const int c = s / kCL;
  float cen[3], r[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    cen[d] = (float)center[3 * c + d];   // exactly representable
    r[d] = reff[3 * a + d];
  }
  const float q = (float)sc.qs[a];
  const size_t Q3 = 3 * (size_t)sc.Q;
  // local coordinates of bead b, as k_local_box32 forms them
  auto local = [&](int b, float* v) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const df A = aligned_df(sc, x32[b * Q3 + 3 * (size_t)a + d], r[d], d);
      const df t = two_sum(A.hi, -cen[d]);
      v[d] = t.hi + (t.lo + A.lo);
    }
  };
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  const int nb = max(N, groups * kBLBeads);
  for (int g = 0; g * kBLBeads < nb; ++g) {
    float v0[3], v1[3];
    const int b0 = g * kBLBeads + lane, b1 = b0 + 32;
    local(min(b0, N - 1), v0);
    local(min(b1, N - 1), v1);
    // the sphere covers the beads 0 .. N-1
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (b0 < N) { lo[d] = fminf(lo[d], v0[d]); hi[d] = fmaxf(hi[d], v0[d]); }
      if (b1 < N) { lo[d] = fminf(lo[d], v1[d]); hi[d] = fmaxf(hi[d], v1[d]); }
    }
    if (g < groups) {
      // rows past n_rows repeat row n_rows - 1
      float w0[3], w1[3];
      if (b0 < n_rows) { w0[0] = v0[0]; w0[1] = v0[1]; w0[2] = v0[2]; } else local(n_rows - 1, w0);
      if (b1 < n_rows) { w1[0] = v1[0]; w1[1] = v1[1]; w1[2] = v1[2]; } else local(n_rows - 1, w1);
      float2* o = xb + ((size_t)g * max_slots + s) * 3 * 32 + lane;
#pragma unroll
      for (int d = 0; d < 3; ++d) o[d * 32] = make_float2(w0[d], w1[d]);
    }
    if (g == 0 && lane == 0) xq[s] = make_float4(v0[0], v0[1], v0[2], q);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  if (lane == 0) {
    ts[s] = sc.type[a];
    float cf[3], h2 = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      cf[d] = 0.5f * (lo[d] + hi[d]);
      const float h = fmaxf(hi[d] - cf[d], cf[d] - lo[d]);
      h2 = fmaf(h, h, h2);
    }
    abox[s] = make_float4(cf[0], cf[1], cf[2], sqrtf(h2) * 1.000001f + (float)margin + 1e-6f);
  }
}

// union bounding box of each cluster over all beads; one warp per cluster, lanes over beads
__global__ void k_cluster_bbox(SysConsts sc, const float* x32, const double* x64, int N, const double* ref,
                               const int* perm, const int* meta, int max_clu, double margin, double* center,
                               float* hext, int* molr, unsigned* emax) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= max_clu || c >= meta[0]) return;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  int atoms[kCL];
#pragma unroll
  for (int k = 0; k < kCL; ++k) atoms[k] = perm[c * kCL + k];
  const size_t Q3 = 3 * (size_t)sc.Q;
  for (int b = lane; b < N; b += 32) {
#pragma unroll
    for (int k = 0; k < kCL; ++k) {
      const int a = atoms[k];
      if (a < 0) continue;
      for (int d = 0; d < 3; ++d) {
        const double v = aligned_coord(coord(x32, x64, b * Q3 + 3 * (size_t)a + d), ref[3 * a + d], sc.L[d],
                                       sc.invL[d]);
        lo[d] = fmin(lo[d], v);
        hi[d] = fmax(hi[d], v);
      }
    }
  }
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  }
  if (lane == 0) {
    int m0 = 0x7fffffff, m1 = -0x7fffffff;
    for (int k = 0; k < kCL; ++k)
      if (atoms[k] >= 0) {
        m0 = min(m0, sc.mol[atoms[k]]);
        m1 = max(m1, sc.mol[atoms[k]]);
      }
    molr[2 * c] = m0;
    molr[2 * c + 1] = m1;
    for (int d = 0; d < 3; ++d) {
      const double cen = (double)(float)(0.5 * (lo[d] + hi[d]));   // exactly representable in FP32
      const double ext = fmax(hi[d] - cen, cen - lo[d]) + margin;
      const float e = __double2float_ru(ext);
      center[3 * c + d] = cen;
      hext[3 * c + d] = e;
      atomicMax(&emax[d], __float_as_uint(e));
    }
  }
}

// cluster-local coordinates of every bead (and the slot types, from bead 1)
template <bool F64>
__global__ void k_local_coords(SysConsts sc, const float* x32, const double* x64, int N, const double* ref,
                               const int* perm, const int* meta, int max_slots, const double* center, float4* xq,
                               double4_32a* xq64, int* ts, float4* eta32, double* eta64) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;   // grid: (slots, beads)
  const int b = blockIdx.y;
  if (s >= meta[0] * kCL) return;
  const int a = perm[s];
  const size_t o = (size_t)b * max_slots + s;            // fixed slot stride
  if (a < 0) {
    const double dmy = (double)kDummyCoord + 3.0 * (s & (kCL - 1));
    if (F64) xq64[o] = make_double4_32a(dmy, dmy, dmy, 0.0);
    else xq[o] = make_float4((float)dmy, (float)dmy, (float)dmy, 0.0f);
    // padding slots have no eta; the pair HVP kernels read it as j-atoms
    eta32[o] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (F64) eta64[3 * o] = eta64[3 * o + 1] = eta64[3 * o + 2] = 0.0;
    if (b == 0) ts[s] = 0;
    return;
  }
  const int c = s / kCL;
  const size_t Q3 = 3 * (size_t)sc.Q;
  double v[3];
  for (int d = 0; d < 3; ++d)
    v[d] = aligned_coord(coord(x32, x64, b * Q3 + 3 * (size_t)a + d), ref[3 * a + d], sc.L[d], sc.invL[d]) -
           center[3 * c + d];
  if (F64) xq64[o] = make_double4_32a(v[0], v[1], v[2], sc.qs[a]);
  else xq[o] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)sc.qs[a]);
  if (b == 0) ts[s] = sc.type[a];
}

__global__ void k_bin_clusters(SysConsts sc, const int* meta, int max_clu, const double* center, const float* hext,
                               int nb0, int nb1, int nb2, double bw0, double bw1, double bw2, double* cwrap,
                               float2* cwdf, float4* cbox, int* cbin, int* bincnt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= max_clu || c >= meta[0]) return;
  int bidx[3];
  const int nb[3] = {nb0, nb1, nb2};
  const double bw[3] = {bw0, bw1, bw2};
  for (int d = 0; d < 3; ++d) {
    double w = center[3 * c + d] - sc.L[d] * floor(center[3 * c + d] * sc.invL[d]);
    if (w >= sc.L[d]) w -= sc.L[d];
    if (w < 0.0) w = 0.0;
    cwrap[3 * c + d] = w;
    const df wd = df_from_double(w);
    cwdf[3 * c + d] = make_float2(wd.hi, wd.lo);
    bidx[d] = (int)fmin(fmax(w / bw[d], 0.0), (double)(nb[d] - 1));
  }
  const int bin = (bidx[0] * nb1 + bidx[1]) * nb2 + bidx[2];
  cbox[2 * c] = make_float4((float)cwrap[3 * c], (float)cwrap[3 * c + 1], (float)cwrap[3 * c + 2], 0.f);
  cbox[2 * c + 1] = make_float4(hext[3 * c], hext[3 * c + 1], hext[3 * c + 2], 0.f);
  cbin[c] = bin;
  atomicAdd(&bincnt[bin], 1);
}

// exclusive scan of n ints (single block); out[n] = total; optional copy to cur; meta slot
__global__ void k_scan(const int* in, int n, int* out, int* cur, int* meta_total) {
  __shared__ int sh[32];
  int carry = 0;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    int tot;
    const int pre = block_excl_scan(v, sh, &tot);
    if (i < n) {
      out[i] = carry + pre;
      if (cur) cur[i] = carry + pre;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    out[n] = carry;
    if (meta_total) *meta_total = carry;
  }
}

__global__ void k_fill_bins(const int* meta, int max_clu, const int* cbin, int* bincur, int* binlist) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= max_clu || c >= meta[0]) return;
  binlist[atomicAdd(&bincur[cbin[c]], 1)] = c;
}

__global__ void k_sort_bins(int nbins, const int* binstart, int* binlist) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const int s = binstart[b], e = binstart[b + 1];
  for (int i = s + 1; i < e; ++i) {
    const int v = binlist[i];
    int j = i - 1;
    while (j >= s && binlist[j] > v) {
      binlist[j + 1] = binlist[j];
      --j;
    }
    binlist[j + 1] = v;
  }
}

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Union over beads of each atom's aligned position, as a sphere (centre relative to the
// cluster centre, radius) used by the exact pruning of cluster pairs.
__global__ void k_atom_box(SysConsts sc, const float* x32, const double* x64, int N, const double* ref,
                           const int* perm, const int* meta, const double* center, double margin, float4* abox) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= meta[0] * kCL) return;
  const int a = perm[s];
  if (a < 0) {
    abox[s] = make_float4(kDummyCoord, kDummyCoord, kDummyCoord, -1.0f);
    return;
  }
  const int c = s / kCL;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  const size_t Q3 = 3 * (size_t)sc.Q;
  for (int b = 0; b < N; ++b)
    for (int d = 0; d < 3; ++d) {
      const double v = aligned_coord(coord(x32, x64, b * Q3 + 3 * (size_t)a + d), ref[3 * a + d], sc.L[d], sc.invL[d]);
      lo[d] = fmin(lo[d], v);
      hi[d] = fmax(hi[d], v);
    }
  float cf[3];
  double r2 = 0.0, e2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double cen = 0.5 * (lo[d] + hi[d]) - center[3 * c + d];
    cf[d] = (float)cen;
    const double h = 0.5 * (hi[d] - lo[d]);
    r2 += h * h;
    const double er = fabs((double)cf[d] - cen);
    e2 += er * er;
  }
  const float r = __double2float_ru(sqrt(r2) + sqrt(e2) + margin + 1e-6);
  abox[s] = make_float4(cf[0], cf[1], cf[2], r);
}

// LJ types of the 8 atoms of each cluster, 4 bits each
__global__ void k_cluster_types(const int* meta, const int* ts, unsigned* ctype) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= meta[0]) return;
  unsigned v = 0;
  for (int k = 0; k < kCL; ++k) v |= ((unsigned)ts[c * kCL + k] & 15u) << (4 * k);
  ctype[c] = v;
}

// Cluster-pair list of one i-cluster per warp.  Candidates come from the bins around the
// i-cluster (every periodic image), pass the union-bounding-box test, then the exact test on
// the atoms' union spheres; bit 29 / bit 30 of an entry mark the j-half-clusters (atoms 0-3 /
// 4-7) that hold at least one pair that can come within rc in some bead.  The union-box test
// runs one candidate per lane; the exact test runs one candidate at a time over the whole warp
// (two atom pairs per lane), and so does the exclusion mask (bit j * 8 + i).  Entries of cluster ci
// go to ent[ci * cap ...] in bin order (deterministic); lcnt[ci] = their number; meta[2] =
// largest count (a count above cap means the list must be rebuilt with a larger cap).
// HALF: every unordered cluster pair once (half-list kernels).  Otherwise every pair from both
// sides.  PM (bead-lane kernels): emask holds the entry's candidate atom pairs (the union
// spheres within reach, exclusions removed, bit j * 8 + i), an entry whose candidates are all
// excluded is dropped, and with HALF the self entry keeps its pairs j > i only.
#ifndef MOP_LIST_MINB
#define MOP_LIST_MINB 6   // 80 registers: 6 blocks (24 warps) per SM hide the latency of the bin walk
#endif
template <bool F64, bool HALF, bool PM>
__global__ void __launch_bounds__(128, MOP_LIST_MINB) k_pair_list(SysConsts sc, const int* meta_in, int max_clu,
                                                   const double* cwrap, const float2* cwdf, const float* hext,
                                                   const unsigned* emax,
                                                   const int* cbin, int nb0, int nb1, int nb2, double bw0, double bw1,
                                                   double bw2, const int* binstart, const int* binlist,
                                                   const int* perm, const int* molr, const float4* abox,
                                                   const float4* cbox, int cap,
                                                   int* lcnt, int4* ent, double4_32a* ent64,
                                                   unsigned long long* emask, int* meta) {
  __shared__ float4 jbox[4][32][kCL];   // per warp: the atom spheres of each lane's candidate
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = blockIdx.x * 4 + warp;
  if (ci >= max_clu || ci >= meta_in[0]) return;   // warp-uniform
  const int iq = lane & 7, jq = lane >> 3;
  const float4 bi4 = abox[ci * kCL + iq];          // this lane's i-atom sphere
  const int ai = perm[ci * kCL + iq];
  const int mol_i = ai >= 0 ? sc.mol[ai] : -1, loc_i = ai >= 0 ? sc.loc[ai] : 0;
  const int nb[3] = {nb0, nb1, nb2};
  const double bw[3] = {bw0, bw1, bw2};
  double wi[3], ei[3];
  float2 widf[3];   // own centre as double-floats (mixed precision)
  int bi[3], R[3];
  const int binc = cbin[ci];
  bi[2] = binc % nb2;
  bi[1] = (binc / nb2) % nb1;
  bi[0] = binc / (nb1 * nb2);
  for (int d = 0; d < 3; ++d) {
    wi[d] = cwrap[3 * ci + d];
    if (!F64) widf[d] = cwdf[3 * ci + d];
    ei[d] = hext[3 * ci + d];
    const double em = __uint_as_float(emax[d]);
    const double reach = fmin(fmax((sc.rc + ei[d] + em) / bw[d] + 1e-6, 0.0), 3.0 * nb[d] + 1.0);
    R[d] = (int)floor(reach) + 1;
  }
  const int mi0 = molr[2 * ci], mi1 = molr[2 * ci + 1];
  const float rcf = (float)sc.rc + 1e-5f;
  const float rcs = (float)sc.rc + 1e-4f, rcs2 = rcs * rcs;
  const float wif[3] = {(float)wi[0], (float)wi[1], (float)wi[2]};
  const float eif[3] = {(float)ei[0], (float)ei[1], (float)ei[2]};
  const float Lf[3] = {sc.Lf[0], sc.Lf[1], sc.Lf[2]};
  const size_t base = (size_t)ci * cap;
  int count = 0;
  for (int dx = -R[0]; dx <= R[0]; ++dx) {
    const int Bx = bi[0] + dx, kx = floor_div(Bx, nb[0]), wx = Bx - kx * nb[0];
    for (int dy = -R[1]; dy <= R[1]; ++dy) {
      const int By = bi[1] + dy, ky = floor_div(By, nb[1]), wy = By - ky * nb[1];
      const int binbase = (wx * nb1 + wy) * nb2;
      // the z window, cut where it crosses a periodic image: each piece is one contiguous
      // range of binlist (bins are ordered with z fastest)
      for (int z0 = bi[2] - R[2]; z0 <= bi[2] + R[2];) {
        const int kz = floor_div(z0, nb[2]);
        const int zl = min(bi[2] + R[2], (kz + 1) * nb[2] - 1);
        const int s0 = binstart[binbase + (z0 - kz * nb[2])];
        const int nbin = binstart[binbase + (zl - kz * nb[2]) + 1] - s0;
        z0 = zl + 1;
        const int kk[3] = {kx, ky, kz};
        // the image shift of this piece in FP32, converted once (not per candidate)
        const float kf[3] = {(float)kx, (float)ky, (float)kz};
        const float kL[3] = {kf[0] * Lf[0], kf[1] * Lf[1], kf[2] * Lf[2]};
        for (int t0 = 0; t0 < nbin; t0 += 32) {
          const int t = t0 + lane;
          int cj = -1;
          bool self = false, own = false;
          double D[3] = {0.0, 0.0, 0.0};
          if (t < nbin) {
            cj = binlist[s0 + t];
            // the owner of an unordered cluster pair (with its image): the parity rule gives each
            // cluster about half of its neighbours
            self = cj == ci && kk[0] == 0 && kk[1] == 0 && kk[2] == 0;
            own = cj != ci ? (((ci ^ cj) & 1) ? ci < cj : ci > cj)
                           : (kk[0] > 0 || (kk[0] == 0 && (kk[1] > 0 || (kk[1] == 0 && kk[2] >= 0))));
            if (HALF && !own) cj = -1;   // half list: owners only
          }
          bool box = false;
          if (cj >= 0) {
            // FP32 pre-test of the union boxes (slack covers the FP32 rounding of the centres)
            const float4 cw = cbox[2 * cj], ce = cbox[2 * cj + 1];
            const float gx = fmaxf(0.f, fabsf(wif[0] - (cw.x + kL[0])) - eif[0] - ce.x);
            const float gy = fmaxf(0.f, fabsf(wif[1] - (cw.y + kL[1])) - eif[1] - ce.y);
            const float gz = fmaxf(0.f, fabsf(wif[2] - (cw.z + kL[2])) - eif[2] - ce.z);
            box = gx * gx + gy * gy + gz * gz < rcs2;
          }
          float Df[3] = {0.f, 0.f, 0.f};   // FP32 Delta for the warp's exact test and the entry
          if (box) {
            for (int d = 0; d < 3; ++d) {
              if (F64) {
                D[d] = wi[d] - (cwrap[3 * cj + d] + kk[d] * sc.L[d]);
                Df[d] = (float)D[d];
              } else {
                // the same difference exactly as a double-float on the FP32 pipes, rounded once:
                // w_i - w_j by TwoSum plus the low parts, minus k L with k Lf exact by an FMA
                const float2 wj = cwdf[3 * cj + d];
                const float p = kL[d];
                df t = two_sum(widf[d].x, -wj.x);
                t = df_add(t, df{-p, (widf[d].y - wj.y) - fmaf(kf[d], sc.Lf[d], -p)});
                Df[d] = t.hi + (t.lo - kf[d] * sc.Llo[d]);
              }
            }
            // the atom spheres of this lane's candidate, read by the whole warp below
#pragma unroll
            for (int j = 0; j < kCL; ++j) jbox[warp][lane][j] = abox[cj * kCL + j];
          }
          __syncwarp();
          // exact test of each surviving candidate by the whole warp, in bin order: lane
          // (i = lane & 7, jq = lane >> 3) tests atom pairs (i, jq) and (i, jq + 4)
          unsigned pend = __ballot_sync(0xffffffffu, box);
          while (pend) {
            const int src = __ffs(pend) - 1;
            pend &= pend - 1;
            const int cs = __shfl_sync(0xffffffffu, cj, src);
            const bool self_s = __shfl_sync(0xffffffffu, (int)self, src) != 0;
            const float Dx = __shfl_sync(0xffffffffu, Df[0], src);
            const float Dy = __shfl_sync(0xffffffffu, Df[1], src);
            const float Dz = __shfl_sync(0xffffffffu, Df[2], src);
            const float4 bj0 = jbox[warp][src][jq], bj1 = jbox[warp][src][jq + 4];
            bool in0 = false, in1 = false;
            if (bi4.w >= 0.f) {
              if (bj0.w >= 0.f) {
                const float ux = bi4.x + Dx - bj0.x, uy = bi4.y + Dy - bj0.y, uz = bi4.z + Dz - bj0.z;
                const float lim = rcf + bi4.w + bj0.w;
                in0 = ux * ux + uy * uy + uz * uz < lim * lim;
              }
              if (bj1.w >= 0.f) {
                const float ux = bi4.x + Dx - bj1.x, uy = bi4.y + Dy - bj1.y, uz = bi4.z + Dz - bj1.z;
                const float lim = rcf + bi4.w + bj1.w;
                in1 = ux * ux + uy * uy + uz * uz < lim * lim;
              }
            }
            const unsigned b0 = __ballot_sync(0xffffffffu, in0), b1 = __ballot_sync(0xffffffffu, in1);
            const unsigned hm = (b0 ? 1u : 0u) | (b1 ? 2u : 0u);
            if (!hm) continue;   // warp-uniform
            unsigned long long pm = 0ull;
            if (PM) {
              // exclusions only matter for clusters whose molecule ranges overlap
              pm = (unsigned long long)b0 | ((unsigned long long)b1 << 32);
              const int mj0 = molr[2 * cs], mj1 = molr[2 * cs + 1];
              if (mi0 <= mj1 && mj0 <= mi1) {
                bool x0 = false, x1 = false;
                if (ai >= 0) {
                  const int a0 = perm[cs * kCL + jq], a1 = perm[cs * kCL + jq + 4];
                  x0 = a0 >= 0 && sc.mol[a0] == mol_i && abs(sc.loc[a0] - loc_i) <= 2;
                  x1 = a1 >= 0 && sc.mol[a1] == mol_i && abs(sc.loc[a1] - loc_i) <= 2;
                }
                pm &= ~((unsigned long long)__ballot_sync(0xffffffffu, x0) |
                        ((unsigned long long)__ballot_sync(0xffffffffu, x1) << 32));
              }
              // a self entry of the half list: each atom pair once (bits j * 8 + i with j > i)
              if (HALF && self_s) pm &= 0x7f3f1f0f07030100ull;
              if (!pm) continue;   // warp-uniform: every candidate pair is excluded
              if (count < cap && lane == src) {
                ent[base + count] = make_int4(cj | (int)(hm << 29) | (self ? kSelfFlag : 0) | (own ? kOwnerFlag : 0),
                                              __float_as_int(Df[0]),
                                              __float_as_int(Df[1]), __float_as_int(Df[2]));
                emask[base + count] = pm;
              }
              ++count;
              continue;
            }
            if (count < cap) {
              // exclusions, bit j * 8 + i (the lane index for j < 4, + 32 for j >= 4); only
              // clusters whose molecule ranges overlap can hold excluded pairs
              unsigned long long m = 0ull;
              const int mj0 = molr[2 * cs], mj1 = molr[2 * cs + 1];
              if (mi0 <= mj1 && mj0 <= mi1) {
                bool x0 = false, x1 = false;
                if (ai >= 0) {
                  const int b0 = perm[cs * kCL + jq], b1 = perm[cs * kCL + jq + 4];
                  x0 = b0 >= 0 && sc.mol[b0] == mol_i && abs(sc.loc[b0] - loc_i) <= 2;
                  x1 = b1 >= 0 && sc.mol[b1] == mol_i && abs(sc.loc[b1] - loc_i) <= 2;
                }
                m = (unsigned long long)__ballot_sync(0xffffffffu, x0) |
                    ((unsigned long long)__ballot_sync(0xffffffffu, x1) << 32);
              }
              if (lane == src) {
                const bool slf = HALF && self;   // the full FP64 list flags no self entry
                const int flags = (int)(hm << 29) | (m ? (int)0x80000000 : 0) | (slf ? kSelfFlag : 0);
                ent[base + count] = make_int4(cj | flags, __float_as_int(Df[0]), __float_as_int(Df[1]),
                                              __float_as_int(Df[2]));
                if (F64) ent64[base + count] = make_double4_32a(D[0], D[1], D[2], 0.0);
                emask[base + count] = m;
              }
            }
            ++count;
          }
          __syncwarp();
        }
      }
    }
  }
  if (lane == 0) {
    lcnt[ci] = min(count, cap);
    atomicMax(&meta[2], count);
    if (count > cap) atomicOr(&meta[3], 1);   // sticky: cleared only by a synchronous rebuild
  }
}

inline int nblk(long long n, int bs) { return (int)((n + bs - 1) / bs); }

// ---- the full list from the owner entries ---------------------------------------------------
// With MOP_LIST_MIRROR the bead-lane full list is built from the half list: the list kernel tests
// every unordered cluster pair once (its owner entry), and the entries of the other side are
// that entry's mirror images.  A mirror entry in cluster cj's list names ci, carries -Delta (the
// list forms Delta as a rounded difference, so the image of cj's own Delta is its exact negation)
// and the candidate mask transposed (bit j 8 + i becomes bit i 8 + j); a self entry gets its
// mask's transpose added (the half list keeps only its pairs j > i).  Each cluster's list is its
// owner entries in bin order, then its mirror entries ordered by (source cluster, position in the
// source list), so the list does not depend on the order of the atomics that place them.
#ifndef MOP_LIST_MIRROR
#define MOP_LIST_MIRROR 1
#endif

// the 8 x 8 bit matrix of m transposed: bit r 8 + c of the result is bit c 8 + r of m (three
// exchanges of off-diagonal blocks of 1, 2 and 4 bits)
__device__ __forceinline__ unsigned long long transpose8x8(unsigned long long m) {
  unsigned long long t = (m ^ (m >> 7)) & 0x00AA00AA00AA00AAull;
  m ^= t ^ (t << 7);
  t = (m ^ (m >> 14)) & 0x0000CCCC0000CCCCull;
  m ^= t ^ (t << 14);
  t = (m ^ (m >> 28)) & 0x00000000F0F0F0F0ull;
  m ^= t ^ (t << 28);
  return m;
}

// one warp per cluster ci over its owner entries: mirror images into the j-clusters' lists at
// lcnt[cj] + (arrival order) with their sort key, self entries completed in place
__global__ void __launch_bounds__(128) k_mirror_fill(const int* meta, int max_clu, int cap, const int* lcnt,
                                                     int4* ent, unsigned long long* emask, int* mcnt, int* ekey) {
  const int lane = threadIdx.x & 31;
  const int ci = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (ci >= max_clu || ci >= meta[0]) return;   // warp-uniform
  const int n = lcnt[ci];
  const size_t base = (size_t)ci * cap;
  for (int k = lane; k < n; k += 32) {
    const int4 E = ent[base + k];
    const unsigned long long m = emask[base + k];
    const unsigned long long mt = transpose8x8(m);
    if (E.x & kSelfFlag) {
      emask[base + k] = m | mt;
      continue;
    }
    const int cj = E.x & kCluMask;
    const int pos = lcnt[cj] + atomicAdd(&mcnt[cj], 1);
    if (pos >= cap) continue;   // counted: k_mirror_sort reports the overflow
    const unsigned hm = ((unsigned)mt ? 1u : 0u) | ((unsigned)(mt >> 32) ? 2u : 0u);
    const size_t d = (size_t)cj * cap + pos;
    ent[d] = make_int4(ci | (int)(hm << 29), __float_as_int(-__int_as_float(E.y)), __float_as_int(-__int_as_float(E.z)),
                       __float_as_int(-__int_as_float(E.w)));
    emask[d] = mt;
    ekey[d] = ci * cap + k;
  }
}

// one warp per cluster: its mirror entries put in key order (rank = number of smaller keys), the
// list count and the largest count (capacity check) updated.  Shared memory: 4 warps x cap x
// (key + entry + mask).
__global__ void __launch_bounds__(128) k_mirror_sort(int* meta, int max_clu, int cap, int* lcnt, int4* ent,
                                                     unsigned long long* emask, const int* mcnt, const int* ekey) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int4* se = reinterpret_cast<int4*>(smem) + (size_t)w * cap;
  unsigned long long* sm = reinterpret_cast<unsigned long long*>(reinterpret_cast<int4*>(smem) + 4 * (size_t)cap) +
                           (size_t)w * cap;
  int* sk = reinterpret_cast<int*>(reinterpret_cast<unsigned long long*>(reinterpret_cast<int4*>(smem) + 4 * (size_t)cap) +
                                   4 * (size_t)cap) + (size_t)w * cap;
  const int c = blockIdx.x * 4 + w;
  if (c >= max_clu || c >= meta[0]) return;   // warp-uniform; no block barrier below
  const int o = lcnt[c], m = mcnt[c];
  const int total = o + m, mm = max(0, min(m, cap - o));
  if (lane == 0) {
    atomicMax(&meta[2], total);
    if (total > cap) atomicOr(&meta[3], 1);
  }
  const size_t base = (size_t)c * cap + o;
  for (int t = lane; t < mm; t += 32) {
    se[t] = ent[base + t];
    sm[t] = emask[base + t];
    sk[t] = ekey[base + t];
  }
  __syncwarp();
  for (int t = lane; t < mm; t += 32) {
    const int key = sk[t];
    int r = 0;
    for (int u = 0; u < mm; ++u) r += sk[u] < key;
    ent[base + r] = se[t];
    emask[base + r] = sm[t];
  }
  __syncwarp();
  if (lane == 0) lcnt[c] = o + mm;
}

// meta[0..3] into mapped host memory (read by the host after the stream synchronises)
__global__ void k_post_meta(const int* meta, int* host_mapped) {
  if (threadIdx.x < 4) reinterpret_cast<volatile int*>(host_mapped)[threadIdx.x] = meta[threadIdx.x];
}

}  // namespace

#define MOP_CK(x)                                          \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_ != cudaSuccess) {                               \
      if (err) *err = std::string(#x) + ": " + cudaGetErrorString(e_); \
      return e_;                                           \
    }                                                      \
  } while (0)
#define MOP_KL()                                          \
  do {                                                    \
    ++*L.counter;                                         \
    MOP_CK(cudaGetLastError());                           \
  } while (0)

namespace {
__global__ void k_max_disp(const float* __restrict__ x, const float* __restrict__ xref, long long n, unsigned* dmax2) {
  __shared__ float sh[8];
  float m = 0.f;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float dx = x[3 * t] - xref[3 * t], dy = x[3 * t + 1] - xref[3 * t + 1], dz = x[3 * t + 2] - xref[3 * t + 2];
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    m = (d2 <= 3.0e38f) ? fmaxf(m, d2) : INFINITY;   // NaN or overflow: force a rebuild
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh[w]);
    atomicMax(dmax2, __float_as_uint(m));   // non-negative floats order like their bits
  }
}
}  // namespace

cudaError_t launch_max_disp(const float* x, const float* xref, long long n, unsigned* dmax2, Launch L) {
  cudaError_t e = cudaMemsetAsync(dmax2, 0, sizeof(unsigned), L.st);
  if (e != cudaSuccess) return e;
  const long long blocks = std::min<long long>((n + 255) / 256, 148LL * 8);
  k_max_disp<<<(int)std::max<long long>(blocks, 1), 256, 0, L.st>>>(x, xref, n, dmax2);
  ++*L.counter;
  return cudaGetLastError();
}

bool bl_direct_coords(const SysConsts& sc) { return sc.precision == 0 && sc.bl != 0 && sc.elec != 1; }

// the cluster-local coordinates, atom spheres and types of the current sort (mixed precision)
cudaError_t local_box32(const SysConsts& sc, const Grid& g, PathHost& P, double margin, Launch L) {
  const int max_slots = g.max_clu * kCL;
  if (bl_direct_coords(sc)) {
    const int n_rows = P.N == 1 ? 1 : P.N - 1;   // the beads that need forces
    cudaError_t e = P.xb.ensure((size_t)bl_groups(n_rows) * max_slots * 3 * 32);
    if (e != cudaSuccess) return e;
    k_local_box32_bl<<<nblk((long long)max_slots * 32, 256), 256, 0, L.st>>>(
        sc, P.x32.p, P.N, n_rows, P.reff.p, P.perm.p, P.meta.p, max_slots, P.center.p, margin, P.xq.p, P.xb.p,
        P.ts.p, P.eta32.p, P.abox.p);
  } else {
    k_local_box32<<<nblk(max_slots, 256), 256, 0, L.st>>>(sc, P.x32.p, P.N, P.reff.p, P.perm.p, P.meta.p, max_slots,
                                                          P.center.p, margin, P.xq.p, P.ts.p, P.eta32.p, P.abox.p);
  }
  ++*L.counter;
  return cudaGetLastError();
}

cudaError_t prep_coords(const SysConsts& sc, const Grid& g, PathHost& P, double margin, Launch L) {
  return local_box32(sc, g, P, margin, L);
}

cudaError_t prep_path(const SysConsts& sc, const Grid& g, PathHost& P, double margin, Launch L, std::string* err,
                      bool sync) {
  const int Q = sc.Q, N = P.N;
  const int ncol = g.ncx * g.ncy;
  const int max_clu = g.max_clu;
  const int max_slots = max_clu * kCL;
  const int nbins = g.nb[0] * g.nb[1] * g.nb[2];
  const bool f64 = sc.precision == 1;
  const float* x32 = f64 ? nullptr : P.x32.p;
  const double* x64 = f64 ? P.x64.p : nullptr;
  cudaStream_t st = L.st;

  MOP_CK(P.ref.ensure(3 * (size_t)Q));
  MOP_CK(P.colid.ensure(Q));
  MOP_CK(P.colcnt.ensure(ncol));
  MOP_CK(P.colinfo.ensure(3 * (size_t)ncol));
  MOP_CK(P.colatoms.ensure(Q));
  MOP_CK(P.perm.ensure(max_slots));
  MOP_CK(P.slot.ensure(Q));
  MOP_CK(P.ts.ensure(max_slots));
  MOP_CK(P.center.ensure(3 * (size_t)max_clu));
  MOP_CK(P.hext.ensure(3 * (size_t)max_clu));
  MOP_CK(P.molr.ensure(2 * (size_t)max_clu));
  MOP_CK(P.emax.ensure(3));
  MOP_CK(P.cbin.ensure(max_clu));
  MOP_CK(P.cwrap.ensure(3 * (size_t)max_clu));
  MOP_CK(P.cwdf.ensure(3 * (size_t)max_clu));
  MOP_CK(P.cbox.ensure(2 * (size_t)max_clu));
  MOP_CK(P.bincnt.ensure(nbins));
  MOP_CK(P.binstart.ensure(nbins + 1));
  MOP_CK(P.bincur.ensure(nbins));
  MOP_CK(P.binlist.ensure(max_clu));
  MOP_CK(P.lcnt.ensure(max_clu));
  MOP_CK(P.abox.ensure(max_slots));
  MOP_CK(P.ctype.ensure(max_clu));
  MOP_CK(P.meta.ensure(4));
  if (f64) MOP_CK(P.xq64.ensure((size_t)N * max_slots));
  else MOP_CK(P.xq.ensure((size_t)N * max_slots));
  MOP_CK(P.eta32.ensure((size_t)N * max_slots));
  if (f64) MOP_CK(P.eta.ensure(3 * (size_t)N * max_slots));

  MOP_CK(cudaMemsetAsync(P.colcnt.p, 0, sizeof(int) * ncol, st));
  MOP_CK(cudaMemsetAsync(P.perm.p, 0xff, sizeof(int) * max_slots, st));
  MOP_CK(cudaMemsetAsync(P.emax.p, 0, sizeof(unsigned) * 3, st));
  MOP_CK(cudaMemsetAsync(P.bincnt.p, 0, sizeof(int) * nbins, st));
  MOP_CK(cudaMemsetAsync(P.meta.p, 0, sizeof(int) * 3, st));   // meta[3] (overflow) is sticky

  const int bs = 256;
  if (!f64) MOP_CK(P.reff.ensure(3 * (size_t)Q));
  k_ref_columns<<<nblk(Q, bs), bs, 0, st>>>(sc, x32, x64, g.ncx, g.ncy, g.wx, g.wy, P.ref.p, f64 ? nullptr : P.reff.p,
                                            P.colid.p, P.colcnt.p);
  MOP_KL();
  k_scan_columns<<<1, 1024, 0, st>>>(P.colcnt.p, ncol, P.colinfo.p, P.meta.p);
  MOP_KL();
  k_fill_columns<<<nblk(Q, bs), bs, 0, st>>>(Q, P.colid.p, P.colinfo.p, P.colatoms.p);
  MOP_KL();
  k_rank<<<ncol, bs, 0, st>>>(P.ref.p, P.colcnt.p, P.colinfo.p, P.colatoms.p, P.perm.p, P.slot.p);
  MOP_KL();
  if (f64) {
    k_cluster_bbox<<<nblk((long long)max_clu * 32, bs), bs, 0, st>>>(sc, x32, x64, N, P.ref.p, P.perm.p, P.meta.p,
                                                                     max_clu, margin, P.center.p, P.hext.p, P.molr.p,
                                                                     P.emax.p);
    MOP_KL();
    k_local_coords<true><<<dim3(nblk(max_slots, bs), N), bs, 0, st>>>(
        sc, x32, x64, N, P.ref.p, P.perm.p, P.meta.p, max_slots, P.center.p, nullptr, P.xq64.p, P.ts.p, P.eta32.p,
        P.eta.p);
    MOP_KL();
  } else {
    k_cluster_bbox32<<<nblk((long long)max_clu * 32, bs), bs, 0, st>>>(sc, x32, N, P.reff.p, P.perm.p, P.meta.p,
                                                                       max_clu, margin, P.center.p, P.hext.p,
                                                                       P.molr.p, P.emax.p);
    MOP_KL();
    MOP_CK(local_box32(sc, g, P, margin, Launch{st, L.counter}));
  }
  k_bin_clusters<<<nblk(max_clu, bs), bs, 0, st>>>(sc, P.meta.p, max_clu, P.center.p, P.hext.p, g.nb[0], g.nb[1],
                                                   g.nb[2], g.bw[0], g.bw[1], g.bw[2], P.cwrap.p, P.cwdf.p, P.cbox.p,
                                                   P.cbin.p, P.bincnt.p);
  MOP_KL();
  k_scan<<<1, 1024, 0, st>>>(P.bincnt.p, nbins, P.binstart.p, P.bincur.p, nullptr);
  MOP_KL();
  k_fill_bins<<<nblk(max_clu, bs), bs, 0, st>>>(P.meta.p, max_clu, P.cbin.p, P.bincur.p, P.binlist.p);
  MOP_KL();
  k_sort_bins<<<nblk(nbins, bs), bs, 0, st>>>(nbins, P.binstart.p, P.binlist.p);
  MOP_KL();
  if (f64) {
    k_atom_box<<<nblk(max_slots, bs), bs, 0, st>>>(sc, x32, x64, N, P.ref.p, P.perm.p, P.meta.p, P.center.p, margin,
                                                    P.abox.p);
    MOP_KL();
  }
  k_cluster_types<<<nblk(max_clu, bs), bs, 0, st>>>(P.meta.p, P.ts.p, P.ctype.p);
  MOP_KL();
  if (!sync && !P.sized) sync = true;   // the first build must size the list on the host
  for (int attempt = 0; attempt < 3; ++attempt) {
    const size_t cap_total = (size_t)max_clu * P.cap;
    MOP_CK(P.ent.ensure(cap_total));
    MOP_CK(P.emask.ensure(cap_total));
    if (f64) MOP_CK(P.ent64.ensure(cap_total));
    if (sync) MOP_CK(cudaMemsetAsync(P.meta.p + 2, 0, 2 * sizeof(int), st));
    const int blocks = nblk(max_clu, 4);
    if (f64)
      k_pair_list<true, false, false><<<blocks, 128, 0, st>>>(sc, P.meta.p, max_clu, P.cwrap.p, P.cwdf.p, P.hext.p, P.emax.p, P.cbin.p,
                                                g.nb[0], g.nb[1], g.nb[2], g.bw[0], g.bw[1], g.bw[2], P.binstart.p,
                                                P.binlist.p, P.perm.p, P.molr.p, P.abox.p, P.cbox.p, P.cap, P.lcnt.p,
                                                P.ent.p, P.ent64.p, P.emask.p, P.meta.p);
    else if (sc.bl == 2)   // bead-lane half list
      k_pair_list<false, true, true><<<blocks, 128, 0, st>>>(sc, P.meta.p, max_clu, P.cwrap.p, P.cwdf.p, P.hext.p, P.emax.p,
                                                             P.cbin.p, g.nb[0], g.nb[1], g.nb[2], g.bw[0], g.bw[1],
                                                             g.bw[2], P.binstart.p, P.binlist.p, P.perm.p, P.molr.p,
                                                             P.abox.p, P.cbox.p, P.cap, P.lcnt.p, P.ent.p, nullptr,
                                                             P.emask.p, P.meta.p);
    else if (sc.bl && MOP_LIST_MIRROR && (size_t)max_clu * P.cap < (1u << 31)) {
      // bead-lane full list: owner entries, then their images (the sort keys ci cap + k are
      // 32-bit; a larger list is built from both sides directly)
      k_pair_list<false, true, true><<<blocks, 128, 0, st>>>(sc, P.meta.p, max_clu, P.cwrap.p, P.cwdf.p, P.hext.p, P.emax.p,
                                                             P.cbin.p, g.nb[0], g.nb[1], g.nb[2], g.bw[0], g.bw[1],
                                                             g.bw[2], P.binstart.p, P.binlist.p, P.perm.p, P.molr.p,
                                                             P.abox.p, P.cbox.p, P.cap, P.lcnt.p, P.ent.p, nullptr,
                                                             P.emask.p, P.meta.p);
      MOP_KL();
      MOP_CK(P.mcnt.ensure(max_clu));
      MOP_CK(P.ekey.ensure((size_t)max_clu * P.cap));
      MOP_CK(cudaMemsetAsync(P.mcnt.p, 0, sizeof(int) * max_clu, st));
      k_mirror_fill<<<blocks, 128, 0, st>>>(P.meta.p, max_clu, P.cap, P.lcnt.p, P.ent.p, P.emask.p, P.mcnt.p, P.ekey.p);
      MOP_KL();
      const size_t sbytes = 4 * (size_t)P.cap * (sizeof(int4) + sizeof(unsigned long long) + sizeof(int));
      if (sbytes > 48 * 1024) MOP_CK(cudaFuncSetAttribute(k_mirror_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sbytes));
      k_mirror_sort<<<blocks, 128, sbytes, st>>>(P.meta.p, max_clu, P.cap, P.lcnt.p, P.ent.p, P.emask.p, P.mcnt.p,
                                                 P.ekey.p);
    } else if (sc.bl)      // bead-lane full list
      k_pair_list<false, false, true><<<blocks, 128, 0, st>>>(sc, P.meta.p, max_clu, P.cwrap.p, P.cwdf.p, P.hext.p, P.emax.p,
                                                        P.cbin.p, g.nb[0], g.nb[1], g.nb[2], g.bw[0], g.bw[1], g.bw[2],
                                                        P.binstart.p, P.binlist.p, P.perm.p, P.molr.p, P.abox.p,
                                                        P.cbox.p, P.cap, P.lcnt.p, P.ent.p, nullptr, P.emask.p,
                                                        P.meta.p);
    else
      k_pair_list<false, true, false><<<blocks, 128, 0, st>>>(sc, P.meta.p, max_clu, P.cwrap.p, P.cwdf.p, P.hext.p, P.emax.p,
                                                       P.cbin.p, g.nb[0], g.nb[1], g.nb[2], g.bw[0], g.bw[1], g.bw[2],
                                                       P.binstart.p, P.binlist.p, P.perm.p, P.molr.p, P.abox.p,
                                                       P.cbox.p, P.cap, P.lcnt.p, P.ent.p, nullptr, P.emask.p,
                                                       P.meta.p);
    MOP_KL();
    if (!sync) return cudaSuccess;   // capture-safe: an overflow shows up in the sticky flag
    MOP_CK(P.mbox.ensure());
    k_post_meta<<<1, 32, 0, st>>>(P.meta.p, P.mbox.d);
    MOP_KL();
    MOP_CK(cudaStreamSynchronize(st));
    int meta[4];
    for (int k = 0; k < 4; ++k) meta[k] = reinterpret_cast<volatile int*>(P.mbox.h)[k];
    P.n_clu = meta[0];
    if (meta[2] <= P.cap) {
      P.max_count = meta[2];
      // keep a quarter of headroom so that later steps (graph replays) rarely overflow
      if (P.max_count + P.max_count / 4 > P.cap) P.cap = (P.max_count + P.max_count / 4 + 31) / 32 * 32;
      else {
        P.sized = true;
        return cudaSuccess;
      }
    } else {
      P.cap = (meta[2] + meta[2] / 4 + 31) / 32 * 32;   // grow and rebuild
    }
  }
  if (err) *err = "pair list did not fit after growing its capacity";
  return cudaErrorMemoryAllocation;
}

}  // namespace mop

