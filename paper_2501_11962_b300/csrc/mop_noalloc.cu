// Allocation-free spring energy.
//
// Some callers cannot allocate device memory at all: code running inside a CUDA-graph capture
// that a host framework replays, plug-ins whose host owns every allocation, or processes that
// must not grow their device footprint after start-up.  mop_spring_energy_noalloc gives them
// the spring energy sum_n sum_i K_i/2 |eta^n_i|^2 (the second term of V_eff) from an eta array
// they already hold.  The reduction is deterministic and fixed-order (FP64 block sums over tiles
// of 256 atoms in caller order, then one block over the tiles), with its block partial sums in a
// fixed, file-scope device array instead of handle memory.  It is not the engine's reduction
// (which sums FP32 terms per warp as double-floats in slot order), so the two agree to rounding
// (about 1e-7 relative), not bit for bit.
//
// The array holds kMaxPartials doubles (512 KiB) on every GPU that loads the library, for the
// life of the process.  All calls share it: calls that overlap on the GPU (different streams
// without ordering, or several host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/mop.h"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxPartials = 65536;
constexpr int kMaxDevices = 64;

// block partial sums, one per (spring, tile of 256 atoms)
static __device__ __align__(256) double g_partials[kMaxPartials];

double* g_partials_addr[kMaxDevices] = {};
std::mutex g_mu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kBlock / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = threadIdx.x < kBlock / 32 ? sh[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) r = warp_sum(r);
  return r;
}

// partials[b] = sum over the atoms of tile t of K_i/2 |eta^n_i|^2, block b = n * tiles + t (one
// grid dimension: n_springs alone may exceed the 65,535 limit of gridDim.y)
__global__ void k_spring_partials(const double* __restrict__ eta, const double* __restrict__ mass, int Q, int tiles,
                                  double k_over_m, double* partials) {
  const size_t n = blockIdx.x / (unsigned)tiles;
  const int i = (int)(blockIdx.x - n * (unsigned)tiles) * kBlock + threadIdx.x;
  double e = 0.0;
  if (i < Q) {
    const double* v = eta + 3 * (n * Q + i);
    e = 0.5 * (mass[i] * k_over_m) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  }
  e = block_sum(e);
  if (threadIdx.x == 0) partials[blockIdx.x] = e;
}

// fixed-order sum of the partials into *out
__global__ void k_sum_partials(const double* partials, int n, double* out) {
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += kBlock) s += partials[k];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace

extern "C" mop_status mop_spring_energy_noalloc(const double* eta, const double* mass, int32_t n_springs,
                                                int32_t n_atoms, double dt_path, double nu_path, double* out,
                                                void* cuda_stream) {
  if (!eta || !mass || !out || n_springs < 0 || n_atoms < 1) return MOP_ERR_ARG;
  if (!std::isfinite(dt_path) || !std::isfinite(nu_path) || !(dt_path > 0) || !(nu_path > 0)) return MOP_ERR_ARG;
  const long long tiles = ((long long)n_atoms + kBlock - 1) / kBlock;
  const long long n_part = tiles * (long long)n_springs;
  if (n_part > kMaxPartials) return MOP_ERR_ARG;   // n_springs * ceil(n_atoms / 256) must be <= 65536
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // Errors of this call are taken from the return values of its own runtime calls, never from
  // cudaGetLastError: an error the caller left pending is neither consumed nor reported as ours.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MOP_ERR_CUDA;
  double* partials = nullptr;
  {
    // first call on this device: resolve the array's device address (host code cannot use its
    // name directly); make this first call outside any stream capture
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return MOP_ERR_CUDA;
      g_partials_addr[dev] = (double*)p;
    }
    partials = g_partials_addr[dev];
  }
  if (n_part > 0) {
    // every partial the sum reads is written by this call, so none needs clearing
    int q = n_atoms, nt = (int)tiles;
    double kom = nu_path / (2.0 * dt_path);
    void* args[] = {(void*)&eta, (void*)&mass, &q, &nt, &kom, &partials};
    if (cudaLaunchKernel((const void*)k_spring_partials, dim3((unsigned)n_part), dim3(kBlock), args, 0, st) !=
        cudaSuccess)
      return MOP_ERR_CUDA;
  }
  int np = (int)n_part;
  void* args2[] = {&partials, &np, &out};
  if (cudaLaunchKernel((const void*)k_sum_partials, dim3(1), dim3(kBlock), args2, 0, st) != cudaSuccess)
    return MOP_ERR_CUDA;
  return MOP_OK;
}
