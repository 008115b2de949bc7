// Host-side state of the engine and the kernel launchers of each translation unit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mop_internal.cuh"

namespace mop {

// Allocation-failure injection for tests, on the host side (no device fault): with the
// environment variable MOP_FAIL_ALLOC = "<call>:<k>[,<call>:<k>...]", the k-th device allocation
// inside the next call of that entry point (mop_create, mop_set_path, mop_veff_and_grad) fails
// once with cudaErrorMemoryAllocation instead of reaching cudaMalloc.  Unset, it does nothing.
void alloc_hook_enter(const char* call);   // at the entry of those calls
bool alloc_hook_fail();                    // true: fail this allocation

// Grow-only device buffer.  ensure() reports allocation failure through its return value.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;  // elements
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = n > 0 ? n : 1;
    cudaError_t e = alloc_hook_fail() ? cudaErrorMemoryAllocation : cudaMalloc(&p, want * sizeof(T));
    if (e != cudaSuccess) { p = nullptr; return e; }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

// Geometry of the spatial sort of one path (host copy, fixed per system).
struct Grid {
  int ncx, ncy;           // columns of the cluster sort
  double wx, wy;          // column widths
  int nb[3];              // bins of the pair search
  double bw[3];           // bin widths
  int max_clu;            // upper bound of the cluster count
};

// page-locked host words that kernels write directly (mapped memory): small results the host
// waits for travel without a copy engine, so they do not queue behind a large download
struct HostMailbox {
  int* h = nullptr;   // host address
  int* d = nullptr;   // device address of the same words
  cudaError_t ensure() {
    if (h) return cudaSuccess;
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&h), 4 * sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&d), h, 0);
    return e;
  }
  ~HostMailbox() {
    if (h) cudaFreeHost(h);
  }
};

struct PathHost {
  bool set = false;
  // mixed precision, FP32 input: the integrator state (x64 from x32, zero velocities) is formed
  // by the first mop_step or mop_kinetic_energy after mop_set_path, not by mop_set_path itself
  bool dyn_stale = false;
  int N = 0;
  int n_clu = 0;
  int cap = 256;          // list entries reserved per i-cluster
  HostMailbox mbox;       // the list counts read after a synchronous build
  int max_count = 0;      // largest list of the last synchronous build
  bool sized = false;     // cap has been checked on the host at least once
  // state
  DevBuf<float> x32;      // [N][Q][3]
  DevBuf<double> x64;     // [N][Q][3] master positions (FP64)
  DevBuf<double> vel;     // [N][Q][3]
  bool have_grad = false; // grad_int holds dV/dR at the current positions
  // sort and clusters
  DevBuf<double> ref;     // [Q][3]
  DevBuf<float> reff;     // [Q][3] the same rounded to FP32 (mixed precision)
  DevBuf<int> colid, colcnt, colinfo, colatoms, perm, slot, ts;
  DevBuf<double> center;  // [max_clu][3]
  DevBuf<float> hext;     // [max_clu][3]
  DevBuf<int> molr;       // [max_clu][2]
  DevBuf<unsigned> emax;  // [3] float bits
  DevBuf<int> cbin, bincnt, binstart, bincur, binlist;
  DevBuf<double> cwrap;   // [max_clu][3]
  DevBuf<float2> cwdf;    // [max_clu][3] the same as double-floats (mixed precision)
  DevBuf<float4> cbox;    // [max_clu][2]: FP32 wrapped centre, half extents
  DevBuf<int> lcnt;
  DevBuf<int> mcnt, ekey;   // mirrored full list: mirror entries per cluster, their sort keys
  DevBuf<float4> abox;    // [max_slots] union sphere of each atom over the beads
  DevBuf<unsigned> ctype; // [max_clu] packed LJ types
  DevBuf<int> meta;       // [4]: clusters, (scan total), largest list, sticky overflow flag
  DevBuf<float4> xq;
  DevBuf<double4_32a> xq64;
  DevBuf<float2> xb, etab;   // bead-lane kernels: transposed coordinates and eta
  DevBuf<unsigned long long> jI;   // bead-lane j-side sums of a pass [G][Qpad][3][2][32]
  DevBuf<int4> ent;
  DevBuf<double4_32a> ent64;
  DevBuf<unsigned long long> emask;
  // fields
  DevBuf<double> Fnb, F, eta, Hnb, Heta, grad_int;
  DevBuf<float4> eta32, etalo;
  DevBuf<unsigned> etamax, gmax;
  DevBuf<unsigned long long> jacc;   // mixed mode: fixed-point j-side sums [N][Qpad][3]
  DevBuf<double> e_pair, diag, veff_int;
  DevBuf<double> e_excl;   // Ewald: bead-1 energy partials of the exclusion corrections
  // graph-mode steps: the integrator state before the replays, restored when a list outgrew its
  // capacity so that the replays can run again with a larger one
  DevBuf<double> snap_x64, snap_vel, snap_grad;
  DevBuf<float> snap_x32;
  long long overflows = 0;  // graph-mode step batches of this path run again after a list overflow
  // Verlet skin: coordinates at the last list build and the largest squared displacement since
  DevBuf<float> xref;
  DevBuf<unsigned> dmax;
  bool list_ok = false;     // the list was built with the skin for the current bead count
  int list_N = 0;
  long long builds = 0, reuses = 0;
  // SPME reciprocal space: fixed-point charge grids, FFT input, spectra, potential grids of the
  // force and HVP passes [beads][grid points], bead-1 energy partials
  DevBuf<unsigned long long> pme_q;
  DevBuf<float> pme_phi, pme_phd;
  DevBuf<float2> pme_c;
  DevBuf<double> pme_e;
  // bias
  std::vector<int> hA, hB;   // the groups of all CVs, concatenated
  int n_cv = 0;
  int cv_a[kMaxCV + 1] = {}, cv_b[kMaxCV + 1] = {};
  int cv_e2e[kMaxCV] = {}, cv_com[kMaxCV] = {};
  double cv_width[kMaxCV] = {};
  int n_gauss = 0;          // Gaussians in gc/gw [kMaxGauss][kMaxCV] and gh [kMaxGauss]
  DevBuf<int> gA, gB;
  DevBuf<double> gc, gh, gw;
};

struct Launch {
  cudaStream_t st;
  int* counter;   // launches issued
};

// --- mop_prep.cu: spatial sort, clusters, local coordinates, cluster-pair list ------------
// sync = false: no host synchronisation (stream-capture safe); reuses the capacity of the last
// synchronous build and records an overflow in meta[3].
cudaError_t prep_path(const SysConsts& sc, const Grid& g, PathHost& P, double margin, Launch L,
                      std::string* err, bool sync);

// Verlet skin (mixed precision): *dmax2 = max over atoms and beads of |x - xref|^2 (float bits;
// +inf for non-finite input), and the cluster-local coordinates of a kept sort and list.
cudaError_t launch_max_disp(const float* x, const float* xref, long long n_atoms_beads, unsigned* dmax2, Launch L);
cudaError_t prep_coords(const SysConsts& sc, const Grid& g, PathHost& P, double margin, Launch L);
// true when the prep kernels write the bead-lane coordinates xb themselves (mixed precision,
// reaction field, bead-lane kernels); xq then holds bead 1 only
bool bl_direct_coords(const SysConsts& sc);

// --- mop_pair.cu: pair kernels over every unit of every path -------------------------------
// mode 0 = force (+ bead-0 energy), 1 = adjoint HVP, 2 = FD HVP.  A unit is one i-cluster for
// pair_beads_per_unit(precision) consecutive beads.
int pair_beads_per_unit(int precision);
// units [u_begin, n_units) only (a bead range of a single path: units are bead-major)
cudaError_t launch_pair(const SysConsts& sc, const PathDev* d_paths, int n_paths, long long n_units,
                        int mode, int num_sms, Launch L, long long u_begin = 0);

cudaError_t launch_count_pairs(const SysConsts& sc, const PathDev* d_paths, int n_paths, long long n_units,
                               unsigned long long* counts, int num_sms, Launch L);

// --- mop_pairb.cu: bead-lane pair kernels (mixed precision, full list with pair masks) ------
// A unit is one i-cluster, or a part of one, for a group of kBLBeads beads: a path has
// ceil(beads / kBLBeads) x n_clu x pairb_units_per_cluster() units, group-major.  mode 0 =
// force, 1 = adjoint HVP, 2 = FD HVP.
int pairb_units_per_cluster();
// e1_clu > 0 (force pass, full list, where pairb_fuses_energy1): the launch also sums the bead-1
// pair energy of clusters 0 .. e1_clu - 1 of every path, in place of launch_energy1
cudaError_t launch_pairb(const SysConsts& sc, const PathDev* d_paths, int n_paths, long long n_units, int mode,
                         Launch L, int e1_clu = 0);
bool pairb_fuses_energy1(const SysConsts& sc);
// bead-1 pair energy of every path into e_pair (one warp per i-cluster); grid over max_clu
cudaError_t launch_energy1(const SysConsts& sc, const PathDev* d_paths, int n_paths, int max_clu, Launch L);
// rows [0, n_valid) of src float4 [rows][Qpad] (x, y, z, *) into the transposed bead-lane
// layout dst float2 [G][Qpad][3][32], G = ceil(n_valid / kBLBeads); beads past n_valid repeat
// bead n_valid - 1
cudaError_t launch_bl_transpose(const float4* src, int n_valid, int Qpad, int max_clu, const int* meta, float2* dst,
                                Launch L);
inline int bl_groups(int beads) { return (beads + kBLBeads - 1) / kBLBeads; }
// bead-lane half list: adds the j-side sums jF of every path's pass (mode 0: into the
// double-float Fnb rows [0, n_force); 1, 2: into the FP32 Hnb rows [0, n_hvp), mode 2 scaled
// by -1 / (2 eps) of each bead like the i-side sums)
cudaError_t launch_bl_combine(const SysConsts& sc, const PathDev* d_paths, const PathDev* h_paths, int n_paths,
                              int mode, Launch L);

// --- mop_path.cu: bonded terms, eta, path gradient, bias, reductions, integrator ----------
// grids: (slot blocks of 256, beads, paths); e_bond gets nbx partials per path, e_spring
// max_beads * nbx partials per path
cudaError_t launch_e1(const SysConsts& sc, const PathDev* d_paths, int n_paths, int max_qpad, int max_beads, Launch L,
                      double* e_bond, int nbx);
// beads [n_begin, n_begin + n_count) (default: all max_beads)
cudaError_t launch_e2(const SysConsts& sc, const PathDev* d_paths, int n_paths, int max_qpad, int max_beads, Launch L,
                      double* e_spring, int nbx, int n_begin = 0, int n_count = -1);
cudaError_t launch_excl(const SysConsts& sc, const PathDev* d_paths, int n_paths, int max_beads, int mode, Launch L,
                        int n_begin = 0, int n_count = -1);
// blocks of bead-1 energy partials launch_excl writes (e_excl)
inline int excl_energy_blocks(const SysConsts& sc) { return sc.n_excl ? (sc.Q + kRedBlock - 1) / kRedBlock : 0; }
cudaError_t launch_deposit(const SysConsts& sc, const PathDev* d_paths, int n_paths, double height, double width,
                           Launch L);
cudaError_t launch_bias(const SysConsts& sc, const PathDev* d_paths, int n_paths, Launch L);
cudaError_t launch_reduce(const SysConsts& sc, const PathDev* d_paths, int n_paths, Launch L,
                          const double* e_bond, int e_bond_stride, int n_e1_blocks,
                          const double* e_spring, int e_spring_stride, int n_e2_blocks);
// --- mop_fft.cu: batched 3-D FFT convolution of the SPME grids --------------------------------
constexpr int kFftMaxStages = 16;
constexpr int kFftMaxLen = 2048;   // grid points per axis (factors 2, 3, 5, 7 only)
// one axis of the transform: its length, radices (8, 4, 2, 3, 5, 7), twiddles exp(-2 pi i k / n)
struct FftAxis {
  int n, nr;
  int radix[kFftMaxStages];
  unsigned magic;   // ceil(2^32 / n): idx / n as a multiply-high
  const float2* tw;
};
// lines of length n a block transforms at once (one per lane): 32, or fewer for long lines
// (about 3,200 complex values per shared-memory buffer), and at most `columns`
inline int fft_lines_per_block(int n, int columns) {
  int l = n > 0 ? 3200 / n - 1 : 1;
  if (l > 32) l = 32;
  if (l > columns) l = columns;
  return l < 1 ? 1 : l;
}
// true when n is a product of 2, 3, 5 and 7
bool fft_factor(int n, int* radix, int* nr);
cudaError_t fft_axis_make(int n, DevBuf<float2>& tw, FftAxis* ax);
// For `beads` grids: q (int64 fixed point, [beads][K1][K2][K3]) -> half spectra c ->
// times theta (energy: bead 0's partials of 1/2 sum theta |F|^2) -> potential out [beads][K1][K2][K3]
cudaError_t launch_fft_convolve(const SysConsts& sc, const FftAxis* ax, const unsigned long long* q, float2* c,
                                float* out, int beads, double* energy, Launch L);

// --- mop_pme.cu: SPME reciprocal space (forces into the j-side sums; mode 1: H eta) ----------
struct PmePlans;
PmePlans* pme_plans_create();
void pme_plans_destroy(PmePlans* p);
// plans for batches of `beads` grids; call outside stream capture
cudaError_t pme_plans_ensure(const SysConsts& sc, PmePlans* plans, int beads, std::string* err);
// mode 0: forces of beads [0, n_force) plus the bead-1 energy partials (pme_e); mode 1: H eta of
// beads [0, n_hvp) (needs the potential grids of mode 0 and eta32)
cudaError_t launch_pme(const SysConsts& sc, const PathDev* d_paths, const PathDev* h_paths, int n_paths,
                       int max_beads, int mode, PmePlans* plans, Launch L, std::string* err);
// blocks of bead-1 energy partials written by launch_pme
// (the blocks of the x-line pass of launch_fft_convolve)
inline int pme_energy_blocks(const SysConsts& sc) {
  if (sc.pme_nk == 0) return 0;
  const int cw = sc.pme_K[1] * sc.pme_kc3, l = fft_lines_per_block(sc.pme_K[0], cw);
  return (cw + l - 1) / l;
}

cudaError_t launch_kick(const SysConsts& sc, double* vel, const double* grad, int N, double half_dt, Launch L);
// the Philox step counter is read from device memory (*step), so a captured step can be replayed
cudaError_t launch_drift(const SysConsts& sc, double* x64, double* vel, float* x32, int N, double dt,
                         double gamma, double kT, uint64_t seed, const unsigned long long* step, Launch L);
cudaError_t launch_step_inc(unsigned long long* step, Launch L);
cudaError_t launch_kinetic(const SysConsts& sc, const double* vel, int N, double* out, Launch L);

}  // namespace mop
