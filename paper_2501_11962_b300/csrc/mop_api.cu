// C ABI of the engine (include/mop.h): handle, validation, uploads, and the order of the
// kernel passes of one evaluation of V_eff and its gradient (Eq. 3, Eqs. 5-7):
//   per path: spatial sort + cluster-pair list (mop_prep.cu)
//   all paths, one launch each: pair force -> bonded + eta -> pair HVP (adjoint or FD) ->
//   bonded HVP + gradient -> bias -> V_eff reduction
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mop.h"
#include "mop_host.h"

using namespace mop;

namespace mop {
constexpr int kCopyChunks = 8;   // bead chunks of the HVP pass whose gradients are copied while later chunks run

namespace failhook {
// MOP_FAIL_ALLOC, parsed once: each "<call>:<k>" fires once per process
struct FailSpec {
  std::string call;
  int k;
  std::atomic<bool> fired{false};
};
std::vector<FailSpec*>& fail_specs() {
  static std::vector<FailSpec*> specs = [] {
    std::vector<FailSpec*> v;
    if (const char* env = getenv("MOP_FAIL_ALLOC")) {
      std::string all(env);
      size_t pos = 0;
      while (pos <= all.size()) {
        const size_t end = std::min(all.find(',', pos), all.size());
        const std::string item = all.substr(pos, end - pos);
        const size_t c = item.find(':');
        if (c != std::string::npos) {
          FailSpec* f = new FailSpec();
          f->call = item.substr(0, c);
          f->k = atoi(item.c_str() + c + 1);
          v.push_back(f);
        }
        pos = end + 1;
      }
    }
    return v;
  }();
  return specs;
}
thread_local const char* t_call = nullptr;
thread_local int t_allocs = 0;
}  // namespace failhook
using failhook::FailSpec;
using failhook::fail_specs;
using failhook::t_call;
using failhook::t_allocs;

void alloc_hook_enter(const char* call) {
  t_call = call;
  t_allocs = 0;
}

// marks the body of an entry point for MOP_FAIL_ALLOC
struct AllocScope {
  explicit AllocScope(const char* call) { alloc_hook_enter(call); }
  ~AllocScope() { alloc_hook_enter(nullptr); }
};

bool alloc_hook_fail() {
  const std::vector<FailSpec*>& v = fail_specs();
  if (v.empty() || !t_call) return false;
  ++t_allocs;
  for (FailSpec* f : v)
    if (f->call == t_call && f->k == t_allocs && !f->fired.exchange(true)) return true;
  return false;
}
}

struct mop_handle {
  int device = 0;
  int num_sms = 148;
  SysConsts sc{};
  Grid grid{};
  int hvp_mode = 0, precision = 0;
  double temperature = 300.0, fd_h = 1e-5;
  std::string err;
  int launches = 0;
  uint64_t step_count = 0;
  // device copies of the system
  DevBuf<double> mass, Kspr, cL, qs;
  DevBuf<float2> c_df;
  DevBuf<float2> K_df;
  DevBuf<int> type, mol, loc, inc_off;
  DevBuf<int4> inc;
  DevBuf<double2> incp;
  DevBuf<float2> incpf;
  DevBuf<float4> tab;
  DevBuf<double4_32a> tab64;
  // paths
  PathHost paths[kMaxPaths];
  DevBuf<PathDev> d_paths, d_one;
  DevBuf<double> e_bond, e_spring, scratch;
  DevBuf<int> excl_off, excl_nb;          // Ewald exclusion partners of every atom (CSR)
  DevBuf<float> pme_theta;                // SPME kernel [K1][K2][K3 / 2 + 1]
  PmePlans* pme = nullptr;                // FFT twiddle tables and axis factorisations
  double skin = 0.0;                      // Verlet skin of the pair lists (0: rebuild every time)
  DevBuf<unsigned long long> counts;
  mop_tuning tuning{1.0, 0.5};
  double box[3] = {0.0, 0.0, 0.0};
  std::vector<int> last_ids;
  std::vector<PathDev> last_pd;
  // instrumentation
  bool profiling = false;
  cudaEvent_t ev[7] = {};
  // gradient copies to pinned host memory overlapped with the HVP pass (mop_veff_and_grad)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t cev[kCopyChunks] = {};
  // asynchronous host calls (MOP_ASYNC): coordinates staged through two device buffers on their
  // own stream, results copied on another while the next evaluation runs
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  DevBuf<unsigned char> stg[2];
  cudaEvent_t stg_ready[2] = {}, stg_free[2] = {};
  bool stg_used[2] = {false, false};
  int stg_next = 0;
  cudaEvent_t d2h_done = nullptr;   // recorded after the last asynchronous result copy
  bool d2h_pending = false;         // that copy reads grad_int / veff_int: E2 waits for it
  // CUDA-graph mode of mop_step
  bool graph_mode = false;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t graph_stream = nullptr;
  std::vector<int> graph_ids;
  double graph_dt = 0.0, graph_gamma = -1.0;
  uint64_t graph_seed = 0;
  DevBuf<unsigned long long> step_dev;   // Philox step counter read by the integrator
  DevBuf<int> flag;                       // non-finite input flag of mop_set_path
  bool step_ready = false;
};

namespace {

mop_status fail(mop_handle* h, mop_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return s;
}

mop_status cuda_fail(mop_handle* h, cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(h, e == cudaErrorMemoryAllocation ? MOP_ERR_OOM : MOP_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(h, x)                                   \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #x); \
  } while (0)

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// precision copies of a path; *bad (if non-NULL) is set when a coordinate is not finite
// coordinates in both precisions; `copy` (may be NULL) receives the input as it is, so that
// device input needs no separate device-to-device copy (which would queue on a copy engine behind
// an asynchronous download)
__global__ void k_f2d(const float* in, float* copy, double* out, long long n, int* bad) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const float v = in[t];
    if (copy) copy[t] = v;
    if (out) out[t] = widen(v);
    if (bad && !isfinite(v)) atomicOr(bad, 1);
  }
}
__global__ void k_d2f(const double* in, double* copy, float* out, long long n, int* bad) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const double v = in[t];
    if (copy) copy[t] = v;
    out[t] = (float)v;
    if (bad && !isfinite(v)) atomicOr(bad, 1);
  }
}

// slot-ordered field -> caller-ordered [N][Q][3], zero rows outside [0, n_rows).
// fmt 0: FP64 x 3; 1: double-float (hi, lo) x 3; 2: float4
// fmt 0: double [rows][Qpad][3]; 1: double-float float2 [rows][Qpad][3]; 2: float4 [rows][Qpad];
// 3: double-float float4 hi [rows][Qpad] plus float4 lo (f2)
__global__ void k_gather_field(const void* f, const float4* f2, int fmt, const int* slot, int Q, int Qpad, int N,
                               int n_rows, double* out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;   // grid: (atoms, beads)
  if (a >= Q) return;
  const int n = blockIdx.y;
  const size_t t = (size_t)n * Q + a;
  const size_t k = (size_t)n * Qpad + slot[a];
  for (int c = 0; c < 3; ++c) {
    double v = 0.0;
    if (n < n_rows) {
      if (fmt == 0) v = ((const double*)f)[3 * k + c];
      else if (fmt == 1) {
        const float2 w = ((const float2*)f)[3 * k + c];
        v = (double)w.x + (double)w.y;
      } else {
        const float4 w = ((const float4*)f)[k];
        v = c == 0 ? w.x : (c == 1 ? w.y : w.z);
        if (fmt == 3) {
          const float4 l = f2[k];
          v += c == 0 ? l.x : (c == 1 ? l.y : l.z);
        }
      }
    }
    out[3 * t + c] = v;
  }
}

inline int nblk(long long n, int bs) { return (int)((n + bs - 1) / bs); }

template <class T>
mop_status upload(mop_handle* h, DevBuf<T>& b, const T* src, size_t n) {
  CK(h, b.ensure(n));
  if (n) CK(h, cudaMemcpy(b.p, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return MOP_OK;
}

// Evaluates the listed paths.  dev_veff/dev_grad: caller device pointers (or NULL for the
// handle's buffers).  Enqueues everything on st; the only host synchronisation is the read of
// the cluster and pair counts in prep_path.
// sync = false makes the call stream-capture safe: no host synchronisation, no allocation (the
// buffers must already have their size from an earlier synchronous call) and no host-to-device
// copy of the path table (it must already be on the device).
// host_grad (pinned host memory, one path, mixed precision, no SPME grid): the HVP pass runs in
// kCopyChunks bead chunks, each followed by its E2, and the finished gradient rows are copied to
// host_grad on a second stream while later chunks compute; *copied is set when that happened.
mop_status evaluate(mop_handle* h, const std::vector<int>& ids, double* dev_veff, double* dev_grad,
                    cudaStream_t st, bool sync = true, double* host_grad = nullptr, bool* copied = nullptr) {
  SysConsts& sc = h->sc;
  Launch L{st, &h->launches};
  const bool fd = h->hvp_mode == MOP_HVP_FD;
  const double margin = fd ? h->fd_h : 0.0;
  std::vector<PathDev> pd(ids.size());
  if (h->profiling) CK(h, cudaEventRecord(h->ev[0], st));
  long long units = 0, units_h = 0;
  int max_qpad = 0, max_nf = 0, max_n = 0;
  size_t goff = 0;
  for (size_t k = 0; k < ids.size(); ++k) {
    PathHost& P = h->paths[ids[k]];
    std::string err;
    // Verlet skin: keep the sort and the list while no atom has moved more than skin / 2
    const bool skin = h->skin > 0.0 && sync && h->precision == MOP_PREC_MIXED;
    bool reuse = false;
    if (skin && P.list_ok && P.list_N == P.N) {
      CK(h, launch_max_disp(P.x32.p, P.xref.p, (long long)P.N * sc.Q, P.dmax.p, L));
      unsigned d2bits = 0;
      CK(h, cudaMemcpyAsync(&d2bits, P.dmax.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      CK(h, cudaStreamSynchronize(st));
      float d2;
      memcpy(&d2, &d2bits, sizeof(d2));
      reuse = (double)d2 < 0.25 * h->skin * h->skin;
    }
    cudaError_t e;
    if (reuse) {
      e = prep_coords(sc, h->grid, P, margin + 0.5 * h->skin, L);
      ++P.reuses;
    } else {
      e = prep_path(sc, h->grid, P, skin ? margin + 0.5 * h->skin : margin, L, &err, sync);
      if (e == cudaSuccess) {
        ++P.builds;
        P.list_ok = false;
        if (skin) {
          CK(h, P.xref.ensure(3 * (size_t)P.N * sc.Q));
          CK(h, P.dmax.ensure(1));
          CK(h, cudaMemcpyAsync(P.xref.p, P.x32.p, sizeof(float) * 3 * (size_t)P.N * sc.Q, cudaMemcpyDeviceToDevice, st));
          P.list_ok = true;
          P.list_N = P.N;
        }
      }
    }
    if (e != cudaSuccess) return fail(h, e == cudaErrorMemoryAllocation ? MOP_ERR_OOM : MOP_ERR_CUDA, "%s", err.c_str());
    const int N = P.N, Qpad = h->grid.max_clu * kCL;   // fixed slot stride (capture safe)
    const int n_force = N == 1 ? 1 : N - 1, n_hvp = N - 1;
    if (sc.bl) {
      // bead-lane kernels read the coordinates with the beads innermost: written so by the prep
      // kernel with the reaction field, transposed from xq otherwise
      CK(h, P.xb.ensure((size_t)bl_groups(n_force) * Qpad * 3 * 32));
      if (!bl_direct_coords(sc)) CK(h, launch_bl_transpose(P.xq.p, n_force, Qpad, h->grid.max_clu, P.meta.p, P.xb.p, L));
      if (n_hvp > 0) CK(h, P.etab.ensure((size_t)bl_groups(n_hvp) * Qpad * 3 * 32));
      // j-side sums: the H eta pass (bl 1, 2) and the force pass of the half list (bl 2)
      const int jrows = sc.bl == 2 ? std::max(n_force, n_hvp) : (sc.bl == 1 ? n_hvp : 0);
      if (jrows > 0) {
        CK(h, P.jI.ensure((size_t)bl_groups(jrows) * Qpad * 3 * 64));
      }
    }
    // j-side sums: the half-list kernels, and the Ewald exclusion and SPME passes
    const bool use_jacc = h->precision == MOP_PREC_MIXED && (!sc.bl || sc.elec == 1);
    const size_t nq3 = 3 * (size_t)N * Qpad;
    CK(h, P.Fnb.ensure(3 * (size_t)n_force * Qpad));
    CK(h, P.F.ensure(nq3));
    if (h->precision == MOP_PREC_FP64) CK(h, P.eta.ensure(nq3));
    CK(h, P.eta32.ensure((size_t)N * Qpad));
    if (h->precision == MOP_PREC_MIXED) CK(h, P.etalo.ensure((size_t)N * Qpad));
    CK(h, P.Hnb.ensure(nq3));
    CK(h, P.Heta.ensure(nq3));
    CK(h, P.etamax.ensure(N));
    CK(h, P.gmax.ensure(N));
    if (use_jacc) CK(h, P.jacc.ensure(nq3));
    CK(h, P.e_pair.ensure(h->grid.max_clu));
    if (sc.elec == 1) CK(h, P.e_excl.ensure(std::max(1, excl_energy_blocks(sc))));
    const bool pme = sc.pme_nk > 0;
    if (pme) {
      const size_t nb = (size_t)std::max(n_force, n_hvp);
      CK(h, P.pme_q.ensure(nb * sc.pme_nk));
      CK(h, P.pme_c.ensure(nb * sc.pme_nkc));
      CK(h, P.pme_phi.ensure((size_t)n_force * sc.pme_nk));
      CK(h, P.pme_phd.ensure(std::max<size_t>(1, (size_t)n_hvp * sc.pme_nk)));
      CK(h, P.pme_e.ensure(pme_energy_blocks(sc)));
      if (sync) {
        std::string perr;
        cudaError_t e = pme_plans_ensure(sc, h->pme, n_force, &perr);
        if (e == cudaSuccess) e = pme_plans_ensure(sc, h->pme, n_hvp, &perr);
        if (e != cudaSuccess) return fail(h, MOP_ERR_OOM, "%s", perr.c_str());
      }
    }
    CK(h, P.diag.ensure(8));
    CK(h, P.veff_int.ensure(1));
    CK(h, P.grad_int.ensure(3 * (size_t)N * sc.Q));
    CK(h, cudaMemsetAsync(P.etamax.p, 0, sizeof(unsigned) * N, st));
    CK(h, cudaMemsetAsync(P.gmax.p, 0, sizeof(unsigned) * N, st));
    PathDev& D = pd[k];
    memset(&D, 0, sizeof(D));
    D.N = N;
    D.n_force = n_force;
    D.n_hvp = n_hvp;
    D.Q = sc.Q;
    D.Qpad = Qpad;
    D.n_clu = h->grid.max_clu;
    D.meta = P.meta.p;
    D.unit_off = units;
    D.unit_off_h = units_h;
    const int bpu = sc.bl ? kBLBeads : pair_beads_per_unit(h->precision);
    const int upc = sc.bl ? pairb_units_per_cluster() : 1;   // units per cluster and bead group
    units += (long long)((n_force + bpu - 1) / bpu) * h->grid.max_clu * upc;
    units_h += (long long)((n_hvp + bpu - 1) / bpu) * h->grid.max_clu * upc;
    max_qpad = std::max(max_qpad, Qpad);
    max_nf = std::max(max_nf, n_force);
    max_n = std::max(max_n, N);
    D.x32 = h->precision == MOP_PREC_FP64 ? nullptr : P.x32.p;
    D.x64 = h->precision == MOP_PREC_FP64 ? P.x64.p : nullptr;
    D.perm = P.perm.p;
    D.slot = P.slot.p;
    D.xq = P.xq.p;
    D.xq64 = P.xq64.p;
    D.ts = P.ts.p;
    D.lcnt = P.lcnt.p;
    D.cap = P.cap;
    D.ctype = P.ctype.p;
    D.ent = P.ent.p;
    D.ent64 = P.ent64.p;
    D.emask = P.emask.p;
    D.Fnb = P.Fnb.p;
    D.F = P.F.p;
    D.eta = P.eta.p;
    D.eta32 = P.eta32.p;
    D.etalo = h->precision == MOP_PREC_MIXED ? P.etalo.p : nullptr;
    D.Hnb = P.Hnb.p;
    D.Heta = P.Heta.p;
    D.etamax = P.etamax.p;
    D.gmax = P.gmax.p;
    D.jacc = use_jacc ? P.jacc.p : nullptr;
    D.xb = sc.bl ? P.xb.p : nullptr;
    D.etab = sc.bl && n_hvp > 0 ? P.etab.p : nullptr;
    D.jI = sc.bl == 1 || sc.bl == 2 ? P.jI.p : nullptr;
    D.e_pair = P.e_pair.p;
    D.e_excl = sc.elec == 1 ? P.e_excl.p : nullptr;
    D.cwdf = P.cwdf.p;
    if (pme) {
      D.pme_q = P.pme_q.p;
      D.pme_c = P.pme_c.p;
      D.pme_phi = P.pme_phi.p;
      D.pme_phd = P.pme_phd.p;
      D.pme_e = P.pme_e.p;
    }
    D.grad = dev_grad ? dev_grad + goff : P.grad_int.p;
    goff += 3 * (size_t)N * sc.Q;
    D.n_cv = P.n_cv;
    D.n_gauss = P.n_gauss;
    for (int q = 0; q <= kMaxCV; ++q) {
      D.cv_a[q] = P.cv_a[q];
      D.cv_b[q] = P.cv_b[q];
    }
    for (int q = 0; q < kMaxCV; ++q) {
      D.cv_e2e[q] = P.cv_e2e[q];
      D.cv_com[q] = P.cv_com[q];
      D.cv_width[q] = P.cv_width[q];
    }
    D.gA = P.gA.p;
    D.gB = P.gB.p;
    D.gc = P.gc.p;
    D.gw = P.gw.p;
    D.gh = P.gh.p;
    D.diag = P.diag.p;
    D.veff_out = dev_veff ? dev_veff + k : P.veff_int.p;
  }
  const int np = (int)ids.size();
  const int nbx = nblk(sc.Q, kRedBlock);   // E1/E2 blocks run over atoms in caller order
  const int sb = nbx, ss = max_n * nbx;
  CK(h, h->e_bond.ensure((size_t)np * sb));
  CK(h, h->e_spring.ensure((size_t)np * ss));
  CK(h, h->d_paths.ensure(np));
  if (sync) CK(h, cudaMemcpyAsync(h->d_paths.p, pd.data(), sizeof(PathDev) * np, cudaMemcpyHostToDevice, st));
  auto mark = [&](int k) { return h->profiling ? cudaEventRecord(h->ev[k], st) : cudaSuccess; };
  // the half-list pair kernels add j-side sums into zeroed fixed-point accumulators
  auto clear_jacc = [&](bool hvp) -> cudaError_t {
    for (const PathDev& D : pd) {
      if (!D.jacc) continue;
      const size_t rows = hvp ? (size_t)D.n_hvp : (size_t)D.n_force;
      if (rows == 0) continue;
      cudaError_t e = cudaMemsetAsync(D.jacc, 0, sizeof(unsigned long long) * 3 * rows * D.Qpad, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // bead-lane passes with j-side sums add them into zeroed buffers, added to the pass's rows after it
  auto clear_jf = [&](bool hvp) -> cudaError_t {
    if (!(hvp ? (sc.bl == 1 || sc.bl == 2) : sc.bl == 2)) return cudaSuccess;
    for (const PathDev& D : pd) {
      const int rows = hvp ? D.n_hvp : D.n_force;
      if (rows == 0) continue;
      cudaError_t e = cudaMemsetAsync(D.jI, 0, sizeof(unsigned long long) * bl_groups(rows) * D.Qpad * 3 * 64, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  CK(h, mark(1));
  CK(h, clear_jacc(false));
  if (sc.bl) {
    CK(h, clear_jf(false));
    const bool fuse_e1 = pairb_fuses_energy1(sc);
    CK(h, launch_pairb(sc, h->d_paths.p, np, units, 0, L, fuse_e1 ? h->grid.max_clu : 0));
    if (sc.bl == 2) CK(h, launch_bl_combine(sc, h->d_paths.p, pd.data(), np, 0, L));
    if (!fuse_e1) CK(h, launch_energy1(sc, h->d_paths.p, np, h->grid.max_clu, L));
  } else {
    CK(h, launch_pair(sc, h->d_paths.p, np, units, 0, h->num_sms, L));
  }
  CK(h, launch_excl(sc, h->d_paths.p, np, max_nf, 0, L));
  std::string perr;
  if (sc.pme_nk > 0) {
    cudaError_t e = launch_pme(sc, h->d_paths.p, pd.data(), np, max_nf, 0, h->pme, L, &perr);
    if (e != cudaSuccess) return fail(h, MOP_ERR_CUDA, "SPME (forces): %s %s", cudaGetErrorString(e), perr.c_str());
  }
  CK(h, mark(2));
  CK(h, launch_e1(sc, h->d_paths.p, np, max_qpad, max_nf, L, h->e_bond.p, nbx));
  if (sc.bl) {
    for (const PathDev& D : pd)
      if (D.n_hvp > 0) CK(h, launch_bl_transpose(D.eta32, D.n_hvp, D.Qpad, D.n_clu, D.meta, const_cast<float2*>(D.etab), L));
  }
  CK(h, mark(3));
  if (copied) *copied = false;
  const bool overlap = host_grad && np == 1 && sync && h->precision == MOP_PREC_MIXED && !sc.bl && sc.pme_nk == 0 &&
                       pd[0].n_hvp >= 2 * kCopyChunks && units_h > 0;
  if (overlap) {
    const PathDev& D = pd[0];
    const int N = D.N, nh = D.n_hvp, pairs = (nh + 1) / 2;   // HVP units come in bead pairs
    if (!h->copy_stream) CK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (auto& e : h->cev)
      if (!e) CK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    bool e2e_cv = false;   // an end-to-end CV puts bias gradient on bead 1 too
    for (int q = 0; q < D.n_cv; ++q) e2e_cv = e2e_cv || D.cv_e2e[q];
    const double* gdev = D.grad;
    const size_t row = 3 * (size_t)sc.Q;
    std::vector<std::pair<int, int>> after_bias;
    CK(h, clear_jacc(true));
    if (h->d2h_pending) CK(h, cudaStreamWaitEvent(st, h->d2h_done, 0));
    for (int c = 0; c < kCopyChunks; ++c) {
      const int p0 = pairs * c / kCopyChunks, p1 = pairs * (c + 1) / kCopyChunks;
      const int b0 = 2 * p0, hb1 = std::min(2 * p1, nh);          // HVP beads of the chunk
      const int b1 = c == kCopyChunks - 1 ? N : 2 * p1;            // E2 beads (the last takes bead N)
      CK(h, launch_pair(sc, h->d_paths.p, 1, (long long)p1 * D.n_clu, fd ? 2 : 1, h->num_sms, L,
                        (long long)p0 * D.n_clu));
      CK(h, launch_excl(sc, h->d_paths.p, 1, max_n, fd ? 2 : 1, L, b0, hb1 - b0));
      CK(h, launch_e2(sc, h->d_paths.p, 1, max_qpad, max_n, L, h->e_spring.p, nbx, b0, b1 - b0));
      // the bias adds to the row of bead N and, for an end-to-end CV, of bead 1: those rows are
      // copied after it, the rest of the chunk now
      CK(h, cudaEventRecord(h->cev[c], st));
      CK(h, cudaStreamWaitEvent(h->copy_stream, h->cev[c], 0));
      int r0 = b0;
      for (int b = b0; b <= b1; ++b) {
        const bool touched = b < b1 && (b == N - 1 || (b == 0 && e2e_cv));
        if (b < b1 && !touched) continue;
        if (b > r0)
          CK(h, cudaMemcpyAsync(host_grad + r0 * row, gdev + r0 * row, sizeof(double) * row * (b - r0),
                                cudaMemcpyDeviceToHost, h->copy_stream));
        if (touched) after_bias.push_back({b, b + 1});
        r0 = b + 1;
      }
    }
    CK(h, mark(4));
    CK(h, mark(5));
    CK(h, launch_bias(sc, h->d_paths.p, np, L));
    CK(h, launch_reduce(sc, h->d_paths.p, np, L, h->e_bond.p, sb, sb, h->e_spring.p, ss, ss));
    CK(h, mark(6));
    for (const auto& r : after_bias)
      CK(h, cudaMemcpyAsync(host_grad + r.first * row, gdev + r.first * row, sizeof(double) * row * (r.second - r.first),
                            cudaMemcpyDeviceToHost, st));
    if (copied) *copied = true;
    for (int id : ids) h->paths[id].have_grad = true;
    h->last_ids = ids;
    h->last_pd = pd;
    return MOP_OK;
  }
  if (units_h > 0) {
    CK(h, clear_jacc(true));
    if (sc.bl) {
      CK(h, clear_jf(true));
      CK(h, launch_pairb(sc, h->d_paths.p, np, units_h, fd ? 2 : 1, L));
      if (sc.bl == 1 || sc.bl == 2) CK(h, launch_bl_combine(sc, h->d_paths.p, pd.data(), np, fd ? 2 : 1, L));
    } else {
      CK(h, launch_pair(sc, h->d_paths.p, np, units_h, fd ? 2 : 1, h->num_sms, L));
    }
    CK(h, launch_excl(sc, h->d_paths.p, np, max_n, fd ? 2 : 1, L));
    if (sc.pme_nk > 0) {
      cudaError_t e = launch_pme(sc, h->d_paths.p, pd.data(), np, max_n, 1, h->pme, L, &perr);
      if (e != cudaSuccess) return fail(h, MOP_ERR_CUDA, "SPME (H eta): %s %s", cudaGetErrorString(e), perr.c_str());
    }
  }
  CK(h, mark(4));
  // an asynchronous copy of the previous results may still be reading the gradient and V_eff
  if (h->d2h_pending) CK(h, cudaStreamWaitEvent(st, h->d2h_done, 0));
  CK(h, launch_e2(sc, h->d_paths.p, np, max_qpad, max_n, L, h->e_spring.p, nbx));
  CK(h, mark(5));
  CK(h, launch_bias(sc, h->d_paths.p, np, L));
  CK(h, launch_reduce(sc, h->d_paths.p, np, L, h->e_bond.p, sb, sb, h->e_spring.p, ss, ss));
  CK(h, mark(6));
  for (int id : ids) h->paths[id].have_grad = dev_grad == nullptr;
  h->last_ids = ids;
  h->last_pd = pd;
  return MOP_OK;
}

void drop_graph(mop_handle* h);

// streams and events of the asynchronous host calls, created on first use
cudaError_t async_streams(mop_handle* h) {
  cudaError_t e = cudaSuccess;
  if (!h->h2d_stream) e = cudaStreamCreateWithFlags(&h->h2d_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !h->d2h_stream) e = cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    if (!h->stg_ready[k]) e = cudaEventCreateWithFlags(&h->stg_ready[k], cudaEventDisableTiming);
    if (e == cudaSuccess && !h->stg_free[k]) e = cudaEventCreateWithFlags(&h->stg_free[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess && !h->d2h_done) e = cudaEventCreateWithFlags(&h->d2h_done, cudaEventDisableTiming);
  return e;
}

// the host waits for the asynchronous result copies (before work that is captured in a graph)
cudaError_t settle_copies(mop_handle* h) {
  if (!h->d2h_pending) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(h->d2h_done);
  if (e == cudaSuccess) h->d2h_pending = false;
  return e;
}

// M_p(t) at the integers t = 0..p-1, by the B-spline recursion
// M_n(x) = (x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)) / (n - 1) from M_2(0) = 0, M_2(1) = 1
std::vector<double> bspline_integers(int p) {
  std::vector<double> M = {0.0, 1.0};
  for (int n = 3; n <= p; ++n) {
    std::vector<double> B(n, 0.0);
    for (int t = 0; t < n; ++t) {
      const double a = t < n - 1 ? M[t] : 0.0, b = t >= 1 ? M[t - 1] : 0.0;
      B[t] = (t * a + (n - t) * b) / (n - 1);
    }
    M = B;
  }
  return M;
}

// SPME grid constants of sc and the reciprocal kernel on the half spectrum [K1][K2][K3 / 2 + 1]:
// theta(m) = exp(-pi^2 |m~|^2 / beta^2) / (pi V |m~|^2) |b1(m1) b2(m2) b3(m3)|^2, m~_d = m_d / L_d
// (m folded to |m| <= K / 2), theta(0) = 0, |b(m)|^2 = 1 / |sum_k M_p(k + 1) exp(2 pi i m k / K)|^2.
// Charges are sqrt(f) q, so f is not part of theta.
std::vector<float> pme_kernel(const mop_system_desc* d, SysConsts* sc) {
  const int p = d->pme_order;
  const std::vector<double> Mi = bspline_integers(p);
  double mod[3][1024];
  for (int a = 0; a < 3; ++a) {
    const int K = d->pme_grid[a];
    sc->pme_K[a] = K;
    const double kl = K / d->box[a];
    const float hi = (float)kl;
    sc->pme_kl[a] = make_float2(hi, (float)(kl - (double)hi));
    for (int m = 0; m < K; ++m) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k + 1 < p; ++k) {
        const double ph = 2.0 * M_PI * (double)m * k / K;
        re += Mi[k + 1] * std::cos(ph);
        im += Mi[k + 1] * std::sin(ph);
      }
      mod[a][m] = 1.0 / (re * re + im * im);
    }
  }
  sc->pme_order = p;
  sc->pme_kc3 = sc->pme_K[2] / 2 + 1;
  sc->pme_nk = (long long)sc->pme_K[0] * sc->pme_K[1] * sc->pme_K[2];
  sc->pme_nkc = (long long)sc->pme_K[0] * sc->pme_K[1] * sc->pme_kc3;
  const double V = d->box[0] * d->box[1] * d->box[2], b2 = d->ew_beta * d->ew_beta;
  std::vector<float> th((size_t)sc->pme_nkc);
  size_t o = 0;
  for (int m1 = 0; m1 < sc->pme_K[0]; ++m1)
    for (int m2 = 0; m2 < sc->pme_K[1]; ++m2)
      for (int m3 = 0; m3 < sc->pme_kc3; ++m3, ++o) {
        const int f[3] = {m1, m2, m3};
        double k2 = 0.0;
        for (int a = 0; a < 3; ++a) {
          const int m = f[a] <= sc->pme_K[a] / 2 ? f[a] : f[a] - sc->pme_K[a];
          const double k = m / d->box[a];
          k2 += k * k;
        }
        th[o] = o == 0 ? 0.f
                       : (float)(std::exp(-M_PI * M_PI * k2 / b2) / (M_PI * V * k2) * mod[0][m1] * mod[1][m2] *
                                 mod[2][m3]);
      }
  return th;
}

// column grid of the cluster sort and bins of the pair search for the current tuning
void make_grid(mop_handle* h) {
  Grid& g = h->grid;
  const double* box = h->box;
  const int Q = h->sc.Q;
  const double vol = box[0] * box[1] * box[2];
  const double w = h->tuning.col_factor * std::cbrt(kCL * vol / Q);
  g.ncx = std::max(1, (int)std::lround(box[0] / w));
  g.ncy = std::max(1, (int)std::lround(box[1] / w));
  g.wx = box[0] / g.ncx;
  g.wy = box[1] / g.ncy;
  g.max_clu = (Q + kCL - 1) / kCL + g.ncx * g.ncy;
  for (int k = 0; k < 3; ++k) {
    g.nb[k] = std::max(1, (int)std::floor(box[k] / (h->tuning.bin_factor * h->sc.rc)));
    g.bw[k] = box[k] / g.nb[k];
  }
}

mop_status select_paths(mop_handle* h, int32_t path_id, std::vector<int>* ids) {
  ids->clear();
  if (path_id >= 0) {
    if (path_id >= kMaxPaths) return fail(h, MOP_ERR_ARG, "path_id %d out of range", path_id);
    if (!h->paths[path_id].set) return fail(h, MOP_ERR_STATE, "path %d was never set", path_id);
    ids->push_back(path_id);
  } else {
    for (int p = 0; p < kMaxPaths; ++p)
      if (h->paths[p].set) ids->push_back(p);
    if (ids->empty()) return fail(h, MOP_ERR_STATE, "no path set");
  }
  return MOP_OK;
}

}  // namespace

extern "C" {

mop_status mop_create(const mop_system_desc* d, int device, mop_handle** out) {
  if (!out) return MOP_ERR_ARG;
  *out = nullptr;
  AllocScope scope("mop_create");
  if (!d) return MOP_ERR_ARG;
  const int Q = d->n_atoms, nt = d->n_types;
  if (Q < 1 || nt < 1 || nt > kMaxTypes) return MOP_ERR_ARG;
  if (!d->type || !d->lj_sigma || !d->lj_eps || !d->charge || !d->mass || !d->mol_id || !d->mol_local)
    return MOP_ERR_ARG;
  if (d->n_bonds < 0 || d->n_angles < 0) return MOP_ERR_ARG;
  if (d->n_bonds > 0 && (!d->bond_ij || !d->bond_r0 || !d->bond_k)) return MOP_ERR_ARG;
  if (d->n_angles > 0 && (!d->angle_ijk || !d->angle_th0 || !d->angle_k)) return MOP_ERR_ARG;
  if (d->cutoff_mode != MOP_SHIFTED_FORCE && d->cutoff_mode != MOP_POT_SHIFT) return MOP_ERR_ARG;
  if (d->hvp_mode != MOP_HVP_ADJOINT && d->hvp_mode != MOP_HVP_FD) return MOP_ERR_ARG;
  if (d->precision != MOP_PREC_MIXED && d->precision != MOP_PREC_FP64) return MOP_ERR_ARG;
  const double scal[] = {d->box[0], d->box[1], d->box[2], d->rc, d->eps_rf, d->dt_path, d->nu_path, d->temperature, d->fd_h};
  if (!finite_all(scal, 9) || !finite_all(d->lj_sigma, nt) || !finite_all(d->lj_eps, nt) ||
      !finite_all(d->charge, Q) || !finite_all(d->mass, Q))
    return MOP_ERR_NONFINITE;
  if (d->n_bonds && (!finite_all(d->bond_r0, d->n_bonds) || !finite_all(d->bond_k, d->n_bonds)))
    return MOP_ERR_NONFINITE;
  if (d->n_angles && (!finite_all(d->angle_th0, d->n_angles) || !finite_all(d->angle_k, d->n_angles)))
    return MOP_ERR_NONFINITE;
  if (d->box[0] <= 0 || d->box[1] <= 0 || d->box[2] <= 0 || d->rc <= 0) return MOP_ERR_BOX;
  if (d->rc >= 0.5 * std::min(d->box[0], std::min(d->box[1], d->box[2]))) return MOP_ERR_BOX;
  if (d->eps_rf < 1.0 || d->dt_path <= 0 || d->nu_path <= 0 || d->temperature < 0) return MOP_ERR_ARG;
  if (d->hvp_mode == MOP_HVP_FD && !(d->fd_h > 0)) return MOP_ERR_ARG;
  if (d->elec != MOP_ELEC_RF && d->elec != MOP_ELEC_PME) return MOP_ERR_ARG;
  if (d->elec == MOP_ELEC_PME) {
    if (d->precision != MOP_PREC_MIXED || !std::isfinite(d->ew_beta) || !(d->ew_beta > 0)) return MOP_ERR_ARG;
    if (d->pme_order < 4 || d->pme_order > 8) return MOP_ERR_ARG;
    const bool none = d->pme_grid[0] == 0 && d->pme_grid[1] == 0 && d->pme_grid[2] == 0;
    for (int k = 0; k < 3 && !none; ++k) {
      if (d->pme_grid[k] < d->pme_order || d->pme_grid[k] > 1024) return MOP_ERR_ARG;
      // the grid's FFT runs radices 2, 3, 4, 5 and 7
      int rad[kFftMaxStages], nr = 0;
      if (!fft_factor(d->pme_grid[k], rad, &nr)) return MOP_ERR_ARG;
      // odd orders: the spline moduli vanish at the Nyquist frequency of an even grid
      if ((d->pme_order & 1) && !(d->pme_grid[k] & 1)) return MOP_ERR_ARG;
    }
    // the FD Hessian-vector product has no reciprocal-space counterpart
    if (!none && d->hvp_mode == MOP_HVP_FD) return MOP_ERR_ARG;
  }
  for (int i = 0; i < Q; ++i)
    if (d->type[i] < 0 || d->type[i] >= nt || !(d->mass[i] > 0)) return MOP_ERR_ARG;
  for (int t = 0; t < nt; ++t)
    if (d->lj_sigma[t] < 0 || d->lj_eps[t] < 0) return MOP_ERR_ARG;
  for (int b = 0; b < d->n_bonds; ++b) {
    const int i = d->bond_ij[2 * b], j = d->bond_ij[2 * b + 1];
    if (i < 0 || j < 0 || i >= Q || j >= Q || i == j) return MOP_ERR_ARG;
  }
  for (int a = 0; a < d->n_angles; ++a) {
    const int i = d->angle_ijk[3 * a], j = d->angle_ijk[3 * a + 1], k = d->angle_ijk[3 * a + 2];
    if (i < 0 || j < 0 || k < 0 || i >= Q || j >= Q || k >= Q || i == j || j == k || i == k) return MOP_ERR_ARG;
  }

  int sms = 0;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return MOP_ERR_CUDA;
  }
  mop_handle* h = new mop_handle();
  h->device = device;
  h->num_sms = sms > 0 ? sms : 148;
  h->hvp_mode = d->hvp_mode;
  h->precision = d->precision;
  h->temperature = d->temperature;
  h->fd_h = d->fd_h;

  SysConsts& sc = h->sc;
  sc.Q = Q;
  sc.n_types = nt;
  sc.cutoff_mode = d->cutoff_mode;
  sc.precision = d->precision;
  sc.hvp_mode = d->hvp_mode;
  // mixed precision runs the bead-lane pair kernels on the full list: the force pass over every
  // entry, the H eta pass over the owner entries with exact j-side sums.  MOP_PAIR_KERNELS=blfull
  // runs every entry in both passes, =blhalf both passes on the half list, =half the earlier
  // half-list kernels (all kept for comparison)
  {
    const char* pk = getenv("MOP_PAIR_KERNELS");
    sc.bl = 0;
    if (d->precision == MOP_PREC_MIXED) {
      if (pk && strcmp(pk, "half") == 0) sc.bl = 0;
      else if (pk && strcmp(pk, "blfull") == 0) sc.bl = 3;
      else if (pk && strcmp(pk, "blhalf") == 0) sc.bl = 2;
      else sc.bl = 1;
    }
  }
  for (int k = 0; k < 3; ++k) {
    sc.L[k] = d->box[k];
    sc.invL[k] = 1.0 / d->box[k];
    sc.Lf[k] = (float)d->box[k];
    sc.halfLf[k] = (float)(0.5 * d->box[k]);
    sc.invLf[k] = (float)(1.0 / d->box[k]);
    sc.Llo[k] = (float)(d->box[k] - (double)sc.Lf[k]);
  }
  const double rc = d->rc;
  const bool shifted = d->cutoff_mode == MOP_SHIFTED_FORCE;
  sc.rc = rc;
  sc.rc2 = rc * rc;
  sc.krf = (d->eps_rf - 1.0) / ((2.0 * d->eps_rf + 1.0) * rc * rc * rc);
  sc.crf = 1.0 / rc + sc.krf * rc * rc;
  sc.k2rf = 2.0 * sc.krf;
  sc.drf = shifted ? (-1.0 / (rc * rc) + 2.0 * sc.krf * rc) : 0.0;
  sc.rcf = (float)sc.rc;
  sc.rc2f = (float)sc.rc2;
  sc.krff = (float)sc.krf;
  sc.crff = (float)sc.crf;
  sc.k2rff = (float)sc.k2rf;
  sc.drff = (float)sc.drf;
  sc.fd_h = d->fd_h;
  sc.elec = d->elec;
  if (d->elec == MOP_ELEC_PME) {
    // real-space Ewald: phi = f qq erfc(beta r)/r with the cutoff modifier; drf = phi'(rc)/(f qq)
    const double b = d->ew_beta, ec = std::erfc(b * rc), gc = 2.0 / std::sqrt(M_PI) * b * std::exp(-b * b * rc * rc);
    sc.krf = sc.crf = sc.k2rf = 0.0;
    sc.krff = sc.crff = sc.k2rff = 0.f;
    sc.drf = shifted ? -(ec / (rc * rc) + gc / rc) : 0.0;
    sc.drff = (float)sc.drf;
    sc.ewb = (float)b;
    sc.ewb2 = (float)(b * b);
    sc.ewc2 = (float)(2.0 / std::sqrt(M_PI) * b);
    sc.ewec = (float)(ec / rc);
    double q2 = 0.0;
    for (int i = 0; i < Q; ++i) q2 += d->charge[i] * d->charge[i];
    sc.e_self = -kCoulombF * b / std::sqrt(M_PI) * q2;
  }
  std::vector<float> theta;
  if (d->elec == MOP_ELEC_PME && d->pme_grid[0] > 0) theta = pme_kernel(d, &sc);

  std::vector<double> Kspr(Q), cL(Q), qs(Q);
  std::vector<float2> c_df(Q);
  std::vector<float2> K_df(Q);
  const double sqf = std::sqrt(kCoulombF);
  for (int i = 0; i < Q; ++i) {
    Kspr[i] = d->mass[i] * d->nu_path / (2.0 * d->dt_path);
    cL[i] = d->dt_path / (d->mass[i] * d->nu_path);
    qs[i] = d->charge[i] * sqf;
    const float ch = (float)cL[i];
    c_df[i] = make_float2(ch, (float)(cL[i] - (double)ch));
    const float kh = (float)Kspr[i];
    K_df[i] = make_float2(kh, (float)(Kspr[i] - (double)kh));
  }
  // type-pair table (Lorentz-Berthelot)
  std::vector<float4> tab(kMaxTypes * kMaxTypes);
  std::vector<double4_32a> tab64(kMaxTypes * kMaxTypes);
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const double sig = 0.5 * (d->lj_sigma[a] + d->lj_sigma[b]);
      const double eps = std::sqrt(d->lj_eps[a] * d->lj_eps[b]);
      const double s6 = std::pow(sig, 6);
      const double c6 = 4.0 * eps * s6, c12 = 4.0 * eps * s6 * s6;
      const double dlj = shifted ? (-12.0 * c12 / std::pow(rc, 13) + 6.0 * c6 / std::pow(rc, 7)) : 0.0;
      const double plj = c12 / std::pow(rc, 12) - c6 / std::pow(rc, 6);
      tab[a * nt + b] = make_float4((float)(12.0 * c12), (float)(6.0 * c6), (float)dlj, (float)plj);
      tab64[a * nt + b] = make_double4_32a(12.0 * c12, 6.0 * c6, dlj, plj);
    }
  // bonded incidence lists
  std::vector<int> cnt(Q + 1, 0);
  for (int b = 0; b < d->n_bonds; ++b) { cnt[d->bond_ij[2 * b]]++; cnt[d->bond_ij[2 * b + 1]]++; }
  for (int a = 0; a < d->n_angles; ++a)
    for (int r = 0; r < 3; ++r) cnt[d->angle_ijk[3 * a + r]]++;
  std::vector<int> off(Q + 1, 0);
  for (int i = 0; i < Q; ++i) off[i + 1] = off[i] + cnt[i];
  std::vector<int4> inc(std::max(off[Q], 1));
  std::vector<double2> incp(std::max(off[Q], 1));
  std::vector<float2> incpf(std::max(off[Q], 1));
  std::vector<int> cur(off.begin(), off.end() - 1);
  for (int b = 0; b < d->n_bonds; ++b) {
    const int i = d->bond_ij[2 * b], j = d->bond_ij[2 * b + 1];
    for (int r = 0; r < 2; ++r) {
      const int a = r == 0 ? i : j;
      inc[cur[a]] = make_int4(0 | (r << 2), i, j, -1);
      incp[cur[a]++] = make_double2(d->bond_r0[b], d->bond_k[b]);
    }
  }
  for (int t = 0; t < d->n_angles; ++t) {
    const int i = d->angle_ijk[3 * t], j = d->angle_ijk[3 * t + 1], k = d->angle_ijk[3 * t + 2];
    for (int r = 0; r < 3; ++r) {
      const int a = r == 0 ? i : (r == 1 ? j : k);
      inc[cur[a]] = make_int4(1 | (r << 2), i, j, k);
      incp[cur[a]++] = make_double2(d->angle_th0[t], d->angle_k[t]);
    }
  }
  for (size_t k = 0; k < incp.size(); ++k) incpf[k] = make_float2((float)incp[k].x, (float)incp[k].y);
  // Ewald: the excluded pairs (same molecule, |local_i - local_j| <= 2), i < j
  std::vector<int2> excl;
  if (d->elec == MOP_ELEC_PME) {
    std::vector<int> order(Q);
    for (int i = 0; i < Q; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d->mol_id[a] < d->mol_id[b]; });
    for (int a0 = 0; a0 < Q;) {
      int a1 = a0;
      while (a1 < Q && d->mol_id[order[a1]] == d->mol_id[order[a0]]) ++a1;
      for (int u = a0; u < a1; ++u)
        for (int v = u + 1; v < a1; ++v) {
          const int i = std::min(order[u], order[v]), j = std::max(order[u], order[v]);
          if (std::abs(d->mol_local[i] - d->mol_local[j]) <= 2) excl.push_back(make_int2(i, j));
        }
      a0 = a1;
    }
    std::sort(excl.begin(), excl.end(), [](int2 a, int2 b) { return a.x != b.x ? a.x < b.x : a.y < b.y; });
  }
  sc.n_excl = (int)excl.size();
  // both directions, each atom's partners in ascending order
  std::vector<int> exoff(Q + 1, 0), exnb(std::max<size_t>(1, 2 * excl.size()));
  for (const int2& e : excl) {
    exoff[e.x + 1]++;
    exoff[e.y + 1]++;
  }
  for (int i = 0; i < Q; ++i) exoff[i + 1] += exoff[i];
  {
    std::vector<std::vector<int>> nb(Q);
    for (const int2& e : excl) {
      nb[e.x].push_back(e.y);
      nb[e.y].push_back(e.x);
    }
    for (int i = 0; i < Q; ++i) {
      std::sort(nb[i].begin(), nb[i].end());
      std::copy(nb[i].begin(), nb[i].end(), exnb.begin() + exoff[i]);
    }
  }
  mop_status s;
  if ((s = upload(h, h->mass, d->mass, Q)) || (s = upload(h, h->Kspr, Kspr.data(), Q)) ||
      (s = upload(h, h->cL, cL.data(), Q)) || (s = upload(h, h->qs, qs.data(), Q)) ||
      (s = upload(h, h->c_df, c_df.data(), Q)) || (s = upload(h, h->K_df, K_df.data(), Q)) ||
      (s = upload(h, h->type, d->type, Q)) || (s = upload(h, h->mol, d->mol_id, Q)) ||
      (s = upload(h, h->loc, d->mol_local, Q)) || (s = upload(h, h->inc_off, off.data(), Q + 1)) ||
      (s = upload(h, h->inc, inc.data(), inc.size())) || (s = upload(h, h->incp, incp.data(), incp.size())) ||
      (s = upload(h, h->incpf, incpf.data(), incpf.size())) ||
      (s = upload(h, h->tab, tab.data(), tab.size())) || (s = upload(h, h->tab64, tab64.data(), tab64.size())) ||
      (s = upload(h, h->excl_off, exoff.data(), exoff.size())) || (s = upload(h, h->excl_nb, exnb.data(), exnb.size())) ||
      (s = upload(h, h->pme_theta, theta.data(), theta.size()))) {
    mop_destroy(h);
    return s;
  }
  sc.mass = h->mass.p;
  sc.Kspr = h->Kspr.p;
  sc.cL = h->cL.p;
  sc.qs = h->qs.p;
  sc.c_df = h->c_df.p;
  sc.K_df = h->K_df.p;
  sc.type = h->type.p;
  sc.mol = h->mol.p;
  sc.loc = h->loc.p;
  sc.inc_off = h->inc_off.p;
  sc.inc = h->inc.p;
  sc.incp = h->incp.p;
  sc.incpf = h->incpf.p;
  sc.tab = h->tab.p;
  sc.tab64 = h->tab64.p;
  sc.excl_off = h->excl_off.p;
  sc.excl_nb = h->excl_nb.p;
  sc.pme_theta = h->pme_theta.p;
  h->pme = pme_plans_create();

  for (int k = 0; k < 3; ++k) h->box[k] = d->box[k];
  make_grid(h);
  *out = h;
  return MOP_OK;
}

mop_status mop_destroy(mop_handle* h) {
  if (!h) return MOP_OK;
  cudaSetDevice(h->device);
  h->mass.release(); h->Kspr.release(); h->cL.release(); h->qs.release(); h->c_df.release(); h->K_df.release();
  h->type.release(); h->mol.release(); h->loc.release(); h->inc_off.release();
  h->inc.release(); h->incp.release(); h->incpf.release(); h->tab.release(); h->tab64.release();
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph_stream) cudaStreamDestroy(h->graph_stream);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  for (auto& e : h->cev)
    if (e) cudaEventDestroy(e);
  if (h->h2d_stream) cudaStreamSynchronize(h->h2d_stream), cudaStreamDestroy(h->h2d_stream);
  if (h->d2h_stream) cudaStreamSynchronize(h->d2h_stream), cudaStreamDestroy(h->d2h_stream);
  for (int k = 0; k < 2; ++k) {
    if (h->stg_ready[k]) cudaEventDestroy(h->stg_ready[k]);
    if (h->stg_free[k]) cudaEventDestroy(h->stg_free[k]);
    h->stg[k].release();
  }
  if (h->d2h_done) cudaEventDestroy(h->d2h_done);
  h->step_dev.release();
  h->d_one.release(); h->counts.release();
  h->d_paths.release(); h->e_bond.release(); h->e_spring.release(); h->scratch.release(); h->excl_off.release(); h->excl_nb.release();
  h->pme_theta.release();
  if (h->pme) pme_plans_destroy(h->pme);
  for (auto& P : h->paths) {
    P.x32.release(); P.x64.release(); P.vel.release(); P.snap_x64.release(); P.snap_vel.release(); P.snap_grad.release(); P.snap_x32.release(); P.ref.release(); P.reff.release(); P.colid.release();
    P.colcnt.release(); P.colinfo.release(); P.colatoms.release(); P.perm.release(); P.slot.release();
    P.ts.release(); P.center.release(); P.hext.release(); P.molr.release(); P.emax.release();
    P.cbin.release(); P.bincnt.release(); P.binstart.release(); P.bincur.release(); P.binlist.release();
    P.cwrap.release(); P.cwdf.release(); P.cbox.release(); P.lcnt.release(); P.mcnt.release(); P.ekey.release(); P.abox.release(); P.ctype.release(); P.meta.release(); P.xq.release();
    P.xq64.release(); P.ent.release(); P.ent64.release(); P.emask.release(); P.Fnb.release();
    P.F.release(); P.eta.release(); P.Hnb.release(); P.Heta.release(); P.grad_int.release();
    P.eta32.release(); P.etalo.release(); P.etamax.release(); P.gmax.release(); P.jI.release(); P.jacc.release(); P.e_excl.release(); P.e_pair.release(); P.diag.release(); P.veff_int.release();
    P.gA.release(); P.gB.release(); P.gc.release(); P.gh.release(); P.gw.release();
  }
  delete h;
  return MOP_OK;
}

mop_status mop_set_path(mop_handle* h, int32_t path_id, int32_t n_beads, const void* xyz, int32_t flags,
                        void* cuda_stream) {
  if (!h) return MOP_ERR_ARG;
  h->err.clear();
  if (path_id < 0 || path_id >= kMaxPaths) return fail(h, MOP_ERR_ARG, "path_id %d out of range", path_id);
  if (n_beads < 1) return fail(h, MOP_ERR_ARG, "n_beads must be >= 1");
  if (!xyz) return fail(h, MOP_ERR_ARG, "xyz is NULL");
  CK(h, cudaSetDevice(h->device));
  AllocScope scope("mop_set_path");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  PathHost& P = h->paths[path_id];
  // until this call succeeds the path holds no valid coordinates (a failure leaves it unset, and
  // every other path of the handle as it was)
  if (P.set) drop_graph(h);
  P.set = false;
  const size_t n = 3 * (size_t)n_beads * h->sc.Q;
  const bool f64 = flags & MOP_INPUT_F64;
  const bool async = !(flags & MOP_DEVPTR) && (flags & MOP_ASYNC);
  CK(h, P.x32.ensure(n));
  CK(h, P.x64.ensure(n));
  CK(h, P.vel.ensure(n));
  if (async) {
    // the host array goes to a staging buffer on the handle's upload stream (two buffers, so the
    // next upload overlaps the evaluation that uses this one); the rest reads it on the device
    CK(h, async_streams(h));
    const int k = h->stg_next;
    h->stg_next ^= 1;
    const size_t bytes = n * (f64 ? sizeof(double) : sizeof(float));
    CK(h, h->stg[k].ensure(bytes));
    if (h->stg_used[k]) CK(h, cudaStreamWaitEvent(h->h2d_stream, h->stg_free[k], 0));
    CK(h, cudaMemcpyAsync(h->stg[k].p, xyz, bytes, cudaMemcpyHostToDevice, h->h2d_stream));
    CK(h, cudaEventRecord(h->stg_ready[k], h->h2d_stream));
    CK(h, cudaStreamWaitEvent(st, h->stg_ready[k], 0));
    xyz = h->stg[k].p;
    h->stg_used[k] = true;
  }
  const bool dev = async || (flags & MOP_DEVPTR);
  // host input is checked for non-finite values on the device, during the precision copy
  int* bad = nullptr;
  if (!dev) {
    CK(h, h->flag.ensure(1));
    CK(h, cudaMemsetAsync(h->flag.p, 0, sizeof(int), st));
    bad = h->flag.p;
  }
  if (f64) {
    P.dyn_stale = false;
    if (!dev) CK(h, cudaMemcpyAsync(P.x64.p, xyz, n * sizeof(double), cudaMemcpyHostToDevice, st));
    k_d2f<<<nblk(n, 256), 256, 0, st>>>(dev ? (const double*)xyz : P.x64.p, dev ? P.x64.p : nullptr, P.x32.p,
                                         (long long)n, bad);
  } else {
    if (!dev) CK(h, cudaMemcpyAsync(P.x32.p, xyz, n * sizeof(float), cudaMemcpyHostToDevice, st));
    // mixed precision evaluates from x32 alone: the FP64 integrator copy waits for the integrator
    P.dyn_stale = h->precision == MOP_PREC_MIXED;
    if (dev && P.dyn_stale && !bad) {
      // device input: a plain copy (the non-finite check is the evaluation's, through V_eff)
      CK(h, cudaMemcpyAsync(P.x32.p, xyz, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    } else {
      k_f2d<<<nblk(n, 256), 256, 0, st>>>(dev ? (const float*)xyz : P.x32.p, dev ? P.x32.p : nullptr,
                                           P.dyn_stale ? nullptr : P.x64.p, (long long)n, bad);
    }
  }
  CK(h, cudaGetLastError());
  if (async) CK(h, cudaEventRecord(h->stg_free[(h->stg_next ^ 1)], st));   // the staging buffer may be reused
  if (!P.dyn_stale) CK(h, cudaMemsetAsync(P.vel.p, 0, n * sizeof(double), st));
  if (!dev) {
    int flag = 0;
    CK(h, cudaMemcpyAsync(&flag, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    if (flag) {
      P.set = false;
      drop_graph(h);
      return fail(h, MOP_ERR_NONFINITE, "non-finite coordinate");
    }
  }
  if (P.N != n_beads) drop_graph(h);
  P.N = n_beads;
  P.set = true;
  P.have_grad = false;
  return MOP_OK;
}

mop_status mop_get_path(mop_handle* h, int32_t path_id, float* xyz, int32_t flags, void* cuda_stream) {
  if (!h) return MOP_ERR_ARG;
  if (!xyz) return fail(h, MOP_ERR_ARG, "xyz is NULL");
  std::vector<int> ids;
  mop_status s = select_paths(h, path_id, &ids);
  if (s || path_id < 0) return s ? s : fail(h, MOP_ERR_ARG, "path_id must be >= 0");
  CK(h, cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  PathHost& P = h->paths[path_id];
  const size_t n = 3 * (size_t)P.N * h->sc.Q;
  CK(h, cudaMemcpyAsync(xyz, P.x32.p, n * sizeof(float), (flags & MOP_DEVPTR) ? cudaMemcpyDeviceToDevice
                                                                                 : cudaMemcpyDeviceToHost, st));
  if (!(flags & MOP_DEVPTR)) CK(h, cudaStreamSynchronize(st));
  return MOP_OK;
}

mop_status mop_veff_and_grad(mop_handle* h, int32_t path_id, double* veff, double* grad, int32_t flags,
                             void* cuda_stream) {
  if (!h) return MOP_ERR_ARG;
  h->err.clear();
  h->launches = 0;
  AllocScope scope("mop_veff_and_grad");
  std::vector<int> ids;
  mop_status s = select_paths(h, path_id, &ids);
  if (s) return s;
  CK(h, cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool dev = flags & MOP_DEVPTR;
  if (!dev && (flags & MOP_ASYNC)) {
    // enqueue the evaluation on st and the result copies on the download stream; they overlap
    // the next call's work, and mop_wait ends them
    CK(h, async_streams(h));
    if ((s = evaluate(h, ids, nullptr, nullptr, st, true))) return s;
    CK(h, cudaEventRecord(h->d2h_done, st));
    CK(h, cudaStreamWaitEvent(h->d2h_stream, h->d2h_done, 0));
    size_t goff = 0;
    for (size_t k = 0; k < ids.size(); ++k) {
      PathHost& P = h->paths[ids[k]];
      if (veff) CK(h, cudaMemcpyAsync(veff + k, P.veff_int.p, sizeof(double), cudaMemcpyDeviceToHost, h->d2h_stream));
      const size_t n = 3 * (size_t)P.N * h->sc.Q;
      if (grad) CK(h, cudaMemcpyAsync(grad + goff, P.grad_int.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->d2h_stream));
      goff += n;
    }
    CK(h, cudaEventRecord(h->d2h_done, h->d2h_stream));
    h->d2h_pending = true;
    return MOP_OK;
  }
  // a pinned host gradient buffer lets the gradient copy overlap the HVP pass (one path)
  double* host_grad = nullptr;
  if (!dev && grad && ids.size() == 1) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, grad) == cudaSuccess && at.type == cudaMemoryTypeHost) host_grad = grad;
    cudaGetLastError();
  }
  bool copied = false;
  s = evaluate(h, ids, dev ? veff : nullptr, dev ? grad : nullptr, st, true, host_grad, &copied);
  if (s) return s;
  if (!dev) {
    size_t goff = 0;
    std::vector<double> v(ids.size());
    for (size_t k = 0; k < ids.size(); ++k) {
      PathHost& P = h->paths[ids[k]];
      CK(h, cudaMemcpyAsync(&v[k], P.veff_int.p, sizeof(double), cudaMemcpyDeviceToHost, st));
      const size_t n = 3 * (size_t)P.N * h->sc.Q;
      if (grad && !copied)
        CK(h, cudaMemcpyAsync(grad + goff, P.grad_int.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
      goff += n;
    }
    CK(h, cudaStreamSynchronize(st));
    if (copied) CK(h, cudaStreamSynchronize(h->copy_stream));
    for (size_t k = 0; k < ids.size(); ++k) {
      if (veff) veff[k] = v[k];
      if (!std::isfinite(v[k])) return fail(h, MOP_ERR_NONFINITE, "V_eff of path %d is not finite", ids[k]);
    }
  }
  return MOP_OK;
}

mop_status mop_get_field(mop_handle* h, int32_t path_id, int32_t field, double* out, int32_t flags,
                         void* cuda_stream) {
  if (!h) return MOP_ERR_ARG;
  if (!out) return fail(h, MOP_ERR_ARG, "out is NULL");
  if (path_id < 0 || path_id >= kMaxPaths) return fail(h, MOP_ERR_ARG, "path_id out of range");
  PathHost& P = h->paths[path_id];
  if (!P.set || P.n_clu == 0 || !P.F.p) return fail(h, MOP_ERR_STATE, "path %d has no evaluation", path_id);
  CK(h, cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int N = P.N, Qpad = h->grid.max_clu * kCL;
  const void* f;
  int rows, fmt;
  const bool mixed = h->precision == MOP_PREC_MIXED;
  switch (field) {
    case MOP_FIELD_FORCE: f = P.F.p; rows = N == 1 ? 1 : N - 1; fmt = mixed ? 1 : 0; break;
    case MOP_FIELD_ETA: f = mixed ? (const void*)P.eta32.p : P.eta.p; rows = N - 1; fmt = mixed ? 3 : 0; break;
    case MOP_FIELD_HETA: f = P.Heta.p; rows = N - 1; fmt = mixed ? 2 : 0; break;
    default: return fail(h, MOP_ERR_ARG, "unknown field %d", field);
  }
  const size_t n = 3 * (size_t)N * h->sc.Q;
  double* dst = out;
  if (!(flags & MOP_DEVPTR)) {
    CK(h, h->scratch.ensure(n));
    dst = h->scratch.p;
  }
  k_gather_field<<<dim3(nblk(h->sc.Q, 256), N), 256, 0, st>>>(f, fmt == 3 ? P.etalo.p : nullptr, fmt, P.slot.p,
                                                                h->sc.Q, Qpad, N, rows, dst);
  CK(h, cudaGetLastError());
  if (!(flags & MOP_DEVPTR)) {
    CK(h, cudaMemcpyAsync(out, dst, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
  }
  return MOP_OK;
}

mop_status mop_get_energies(mop_handle* h, int32_t path_id, double out[4]) {
  if (!h) return MOP_ERR_ARG;
  if (!out) return fail(h, MOP_ERR_ARG, "out is NULL");
  if (path_id < 0 || path_id >= kMaxPaths) return fail(h, MOP_ERR_ARG, "path_id out of range");
  PathHost& P = h->paths[path_id];
  if (!P.set || !P.diag.p) return fail(h, MOP_ERR_STATE, "path %d has no evaluation", path_id);
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaDeviceSynchronize());
  CK(h, cudaMemcpy(out, P.diag.p, 4 * sizeof(double), cudaMemcpyDeviceToHost));
  return MOP_OK;
}

}  // extern "C"

namespace {

// validates a group pair against the system
mop_status check_groups(mop_handle* h, const int32_t* grpA, int32_t nA, const int32_t* grpB, int32_t nB) {
  if (!grpA || !grpB || nA < 1 || nB < 1 || nA > kMaxGroup || nB > kMaxGroup)
    return fail(h, MOP_ERR_ARG, "groups need 1..%d atoms each", kMaxGroup);
  for (int k = 0; k < nA; ++k)
    if (grpA[k] < 0 || grpA[k] >= h->sc.Q) return fail(h, MOP_ERR_ARG, "group A index out of range");
  for (int k = 0; k < nB; ++k)
    if (grpB[k] < 0 || grpB[k] >= h->sc.Q) return fail(h, MOP_ERR_ARG, "group B index out of range");
  return MOP_OK;
}

// appends CV number P.n_cv (host copy, then the concatenated groups to the device)
mop_status push_cv(mop_handle* h, PathHost& P, const int32_t* grpA, int32_t nA, const int32_t* grpB, int32_t nB,
                   int32_t flags, double width) {
  const int q = P.n_cv;
  P.hA.insert(P.hA.end(), grpA, grpA + nA);
  P.hB.insert(P.hB.end(), grpB, grpB + nB);
  P.cv_a[q + 1] = (int)P.hA.size();
  P.cv_b[q + 1] = (int)P.hB.size();
  P.cv_e2e[q] = (flags & MOP_E2E) ? 1 : 0;
  P.cv_com[q] = (flags & MOP_COM) ? 1 : 0;
  P.cv_width[q] = width;
  P.n_cv = q + 1;
  mop_status s;
  if ((s = upload(h, P.gA, P.hA.data(), P.hA.size())) || (s = upload(h, P.gB, P.hB.data(), P.hB.size()))) return s;
  P.have_grad = false;
  return MOP_OK;
}

mop_status ensure_gaussians(mop_handle* h, PathHost& P) {
  CK(h, P.gc.ensure((size_t)kMaxGauss * kMaxCV));
  CK(h, P.gw.ensure((size_t)kMaxGauss * kMaxCV));
  CK(h, P.gh.ensure(kMaxGauss));
  return MOP_OK;
}

// appends one Gaussian with n_cv centres and widths (host arrays)
mop_status push_gaussian(mop_handle* h, PathHost& P, double height, const double* centers, const double* widths) {
  if (P.n_gauss >= kMaxGauss) return fail(h, MOP_ERR_ARG, "more than %d Gaussians", kMaxGauss);
  mop_status s = ensure_gaussians(h, P);
  if (s) return s;
  const size_t row = (size_t)P.n_gauss * kMaxCV;
  CK(h, cudaDeviceSynchronize());
  CK(h, cudaMemcpy(P.gc.p + row, centers, sizeof(double) * P.n_cv, cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(P.gw.p + row, widths, sizeof(double) * P.n_cv, cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(P.gh.p + P.n_gauss, &height, sizeof(double), cudaMemcpyHostToDevice));
  ++P.n_gauss;
  P.have_grad = false;
  return MOP_OK;
}

}  // namespace

extern "C" {

mop_status mop_add_bias(mop_handle* h, const int32_t* grpA, int32_t nA, const int32_t* grpB, int32_t nB,
                        double s_center, double height, double width, int32_t path_id, int32_t flags) {
  if (!h) return MOP_ERR_ARG;
  h->err.clear();
  if (path_id < 0 || path_id >= kMaxPaths) return fail(h, MOP_ERR_ARG, "path_id out of range");
  if (!std::isfinite(s_center) || !std::isfinite(height) || !std::isfinite(width))
    return fail(h, MOP_ERR_NONFINITE, "non-finite Gaussian parameter");
  if (!(width > 0)) return fail(h, MOP_ERR_ARG, "width must be > 0");
  CK(h, cudaSetDevice(h->device));
  PathHost& P = h->paths[path_id];
  mop_status s;
  if (grpA || grpB) {
    if ((s = check_groups(h, grpA, nA, grpB, nB))) return s;
    if (P.n_gauss > 0 && P.n_cv != 1)
      return fail(h, MOP_ERR_STATE, "path %d holds Gaussians on %d CVs", path_id, P.n_cv);
    // the single CV of this call replaces the path's CVs (its Gaussians are kept)
    P.hA.clear();
    P.hB.clear();
    P.n_cv = 0;
    if ((s = push_cv(h, P, grpA, nA, grpB, nB, flags, 0.0))) return s;
  } else if (P.n_cv == 0) {
    return fail(h, MOP_ERR_STATE, "no CV groups defined for path %d", path_id);
  } else if (P.n_cv != 1) {
    return fail(h, MOP_ERR_STATE, "path %d has %d CVs: use mop_add_gaussian", path_id, P.n_cv);
  }
  return push_gaussian(h, P, height, &s_center, &width);
}

mop_status mop_add_cv(mop_handle* h, int32_t path_id, const int32_t* grpA, int32_t nA, const int32_t* grpB,
                      int32_t nB, int32_t flags, double deposit_width, int32_t* index) {
  if (!h) return MOP_ERR_ARG;
  h->err.clear();
  if (path_id < 0 || path_id >= kMaxPaths) return fail(h, MOP_ERR_ARG, "path_id out of range");
  if (!std::isfinite(deposit_width) || deposit_width < 0) return fail(h, MOP_ERR_ARG, "invalid deposit width");
  PathHost& P = h->paths[path_id];
  if (P.n_cv >= kMaxCV) return fail(h, MOP_ERR_ARG, "at most %d CVs per path", kMaxCV);
  if (P.n_gauss > 0) return fail(h, MOP_ERR_STATE, "path %d already holds Gaussians", path_id);
  mop_status s = check_groups(h, grpA, nA, grpB, nB);
  if (s) return s;
  CK(h, cudaSetDevice(h->device));
  if ((s = push_cv(h, P, grpA, nA, grpB, nB, flags, deposit_width))) return s;
  if (index) *index = P.n_cv - 1;
  return MOP_OK;
}

mop_status mop_add_gaussian(mop_handle* h, int32_t path_id, double height, const double* centers,
                            const double* widths) {
  if (!h) return MOP_ERR_ARG;
  h->err.clear();
  if (path_id < 0 || path_id >= kMaxPaths || !centers || !widths) return fail(h, MOP_ERR_ARG, "invalid argument");
  PathHost& P = h->paths[path_id];
  if (P.n_cv == 0) return fail(h, MOP_ERR_STATE, "no CVs defined for path %d", path_id);
  if (!std::isfinite(height)) return fail(h, MOP_ERR_NONFINITE, "non-finite Gaussian parameter");
  for (int q = 0; q < P.n_cv; ++q) {
    if (!std::isfinite(centers[q]) || !std::isfinite(widths[q]))
      return fail(h, MOP_ERR_NONFINITE, "non-finite Gaussian parameter");
    if (!(widths[q] > 0)) return fail(h, MOP_ERR_ARG, "widths must be > 0");
  }
  CK(h, cudaSetDevice(h->device));
  return push_gaussian(h, P, height, centers, widths);
}

}  // extern "C"

namespace {

// the integrator state of paths whose mop_set_path deferred it: x64 = x32 widened, velocities 0
mop_status ensure_dynamics(mop_handle* h, const std::vector<int>& ids, cudaStream_t st) {
  for (int id : ids) {
    PathHost& P = h->paths[id];
    if (!P.dyn_stale) continue;
    const size_t n = 3 * (size_t)P.N * h->sc.Q;
    k_f2d<<<nblk(n, 256), 256, 0, st>>>(P.x32.p, nullptr, P.x64.p, (long long)n, nullptr);
    CK(h, cudaGetLastError());
    ++h->launches;
    CK(h, cudaMemsetAsync(P.vel.p, 0, n * sizeof(double), st));
    P.dyn_stale = false;
  }
  return MOP_OK;
}

// one MD step of every listed path: B (half kick), A O A (drift with Langevin noise), evaluation
// of dV_eff/dR at the new positions, B; then the Philox step counter advances
mop_status step_body(mop_handle* h, const std::vector<int>& ids, double dt_md, double gamma, uint64_t seed,
                     cudaStream_t st, bool sync) {
  Launch L{st, &h->launches};
  const double kT = kBoltz * h->temperature;
  for (int id : ids) {
    PathHost& P = h->paths[id];
    CK(h, launch_kick(h->sc, P.vel.p, P.grad_int.p, P.N, 0.5 * dt_md, L));
    CK(h, launch_drift(h->sc, P.x64.p, P.vel.p, P.x32.p, P.N, dt_md, gamma, kT, seed, h->step_dev.p, L));
  }
  mop_status s = evaluate(h, ids, nullptr, nullptr, st, sync);
  if (s) return s;
  for (int id : ids) {
    PathHost& P = h->paths[id];
    CK(h, launch_kick(h->sc, P.vel.p, P.grad_int.p, P.N, 0.5 * dt_md, L));
  }
  CK(h, launch_step_inc(h->step_dev.p, L));
  return MOP_OK;
}

void drop_graph(mop_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  h->graph_exec = nullptr;
}

}  // namespace

extern "C" {

mop_status mop_wait(mop_handle* h) {
  if (!h) return MOP_ERR_ARG;
  CK(h, cudaSetDevice(h->device));
  if (h->h2d_stream) CK(h, cudaStreamSynchronize(h->h2d_stream));
  if (h->d2h_stream) CK(h, cudaStreamSynchronize(h->d2h_stream));
  h->d2h_pending = false;
  return MOP_OK;
}

mop_status mop_step(mop_handle* h, int32_t n_steps, double dt_md, double gamma, uint64_t seed, void* cuda_stream) {
  if (!h) return MOP_ERR_ARG;
  h->err.clear();
  if (n_steps < 0 || !(dt_md > 0) || !(gamma >= 0) || !std::isfinite(dt_md) || !std::isfinite(gamma))
    return fail(h, MOP_ERR_ARG, "invalid step parameters");
  std::vector<int> ids;
  mop_status s = select_paths(h, -1, &ids);
  if (s) return s;
  CK(h, cudaSetDevice(h->device));
  CK(h, settle_copies(h));   // no captured step waits on an asynchronous copy
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if ((s = ensure_dynamics(h, ids, st))) return s;
  CK(h, h->step_dev.ensure(1));
  if (!h->step_ready) {
    CK(h, cudaMemsetAsync(h->step_dev.p, 0, sizeof(unsigned long long), st));
    h->step_ready = true;
  }
  // the first evaluation at the current positions is synchronous: it sizes the pair lists
  bool need = false;
  for (int id : ids) need |= !h->paths[id].have_grad;
  if (need && (s = evaluate(h, ids, nullptr, nullptr, st))) return s;
  if (!h->graph_mode) {
    for (int k = 0; k < n_steps; ++k)
      if ((s = step_body(h, ids, dt_md, gamma, seed, st, true))) return s;
    CK(h, cudaStreamSynchronize(st));
    return MOP_OK;
  }
  // graph mode: capture one step (on a stream of the handle; capture is not allowed on the
  // legacy default stream) and replay it n_steps times
  if (!h->graph_stream) CK(h, cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking));
  CK(h, cudaStreamSynchronize(st));
  cudaStream_t gs = h->graph_stream;
  if (!h->graph_exec || ids != h->graph_ids || dt_md != h->graph_dt || gamma != h->graph_gamma ||
      seed != h->graph_seed) {
    drop_graph(h);
    // a synchronous evaluation uploads the path table the captured step reuses
    if ((s = evaluate(h, ids, nullptr, nullptr, gs))) return s;
    CK(h, cudaStreamSynchronize(gs));
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    s = step_body(h, ids, dt_md, gamma, seed, gs, false);
    cudaError_t ce = cudaStreamEndCapture(gs, &g);
    if (s) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    CK(h, ce);
    ce = cudaGraphInstantiate(&h->graph_exec, g, 0);
    cudaGraphDestroy(g);
    CK(h, ce);
    h->graph_ids = ids;
    h->graph_dt = dt_md;
    h->graph_gamma = gamma;
    h->graph_seed = seed;
  }
  // The replays rebuild every list on the device with the capacity of the last synchronous build
  // (25% headroom).  A list that outgrows it sets a sticky flag and invalidates the replayed
  // steps: the integrator state is then restored from a snapshot taken here, the capacity grows
  // to 1.25 x the largest count the replays met and at least doubles (the replays after an
  // overflow miss pairs, so their counts can fall short of what the true steps need), and the
  // steps run again (at most 4 attempts).
  for (int id : ids) {
    PathHost& P = h->paths[id];
    const size_t n = 3 * (size_t)P.N * h->sc.Q;
    CK(h, P.snap_x64.ensure(n));
    CK(h, P.snap_vel.ensure(n));
    CK(h, P.snap_grad.ensure(n));
    CK(h, P.snap_x32.ensure(n));
    CK(h, cudaMemcpyAsync(P.snap_x64.p, P.x64.p, n * sizeof(double), cudaMemcpyDeviceToDevice, gs));
    CK(h, cudaMemcpyAsync(P.snap_vel.p, P.vel.p, n * sizeof(double), cudaMemcpyDeviceToDevice, gs));
    CK(h, cudaMemcpyAsync(P.snap_grad.p, P.grad_int.p, n * sizeof(double), cudaMemcpyDeviceToDevice, gs));
    CK(h, cudaMemcpyAsync(P.snap_x32.p, P.x32.p, n * sizeof(float), cudaMemcpyDeviceToDevice, gs));
  }
  unsigned long long step0 = 0;
  CK(h, cudaMemcpyAsync(&step0, h->step_dev.p, sizeof(step0), cudaMemcpyDeviceToHost, gs));
  CK(h, cudaStreamSynchronize(gs));
  for (int attempt = 0;; ++attempt) {
    for (int k = 0; k < n_steps; ++k) CK(h, cudaGraphLaunch(h->graph_exec, gs));
    CK(h, cudaStreamSynchronize(gs));
    bool over = false;
    for (int id : ids) {
      PathHost& P = h->paths[id];
      int meta[4];
      CK(h, cudaMemcpy(meta, P.meta.p, sizeof(meta), cudaMemcpyDeviceToHost));
      if (!meta[3]) continue;
      over = true;
      ++P.overflows;
      P.cap = std::max(2 * P.cap, (meta[2] + meta[2] / 4 + 31) / 32 * 32);
      P.sized = false;
      CK(h, cudaMemset(P.meta.p + 3, 0, sizeof(int)));
    }
    if (!over) break;
    drop_graph(h);
    if (attempt == 3)
      return fail(h, MOP_ERR_STATE,
                  "pair lists kept outgrowing their capacity during graph replay; steps since the last "
                  "synchronous call are invalid (set the paths again)");
    for (int id : ids) {
      PathHost& P = h->paths[id];
      const size_t n = 3 * (size_t)P.N * h->sc.Q;
      CK(h, cudaMemcpyAsync(P.x64.p, P.snap_x64.p, n * sizeof(double), cudaMemcpyDeviceToDevice, gs));
      CK(h, cudaMemcpyAsync(P.vel.p, P.snap_vel.p, n * sizeof(double), cudaMemcpyDeviceToDevice, gs));
      CK(h, cudaMemcpyAsync(P.grad_int.p, P.snap_grad.p, n * sizeof(double), cudaMemcpyDeviceToDevice, gs));
      CK(h, cudaMemcpyAsync(P.x32.p, P.snap_x32.p, n * sizeof(float), cudaMemcpyDeviceToDevice, gs));
    }
    CK(h, cudaMemcpyAsync(h->step_dev.p, &step0, sizeof(step0), cudaMemcpyHostToDevice, gs));
    // a synchronous evaluation at the restored positions sizes the lists with the new capacity
    // and uploads the path table; then the step is captured again
    if ((s = evaluate(h, ids, nullptr, nullptr, gs))) return s;
    CK(h, cudaStreamSynchronize(gs));
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    s = step_body(h, ids, dt_md, gamma, seed, gs, false);
    cudaError_t ce = cudaStreamEndCapture(gs, &g);
    if (s) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    CK(h, ce);
    ce = cudaGraphInstantiate(&h->graph_exec, g, 0);
    cudaGraphDestroy(g);
    CK(h, ce);
  }
  return MOP_OK;
}

mop_status mop_set_tuning(mop_handle* h, const mop_tuning* t) {
  if (!h || !t) return MOP_ERR_ARG;
  if (!(t->col_factor >= 0.25 && t->col_factor <= 4.0) || !(t->bin_factor >= 0.2 && t->bin_factor <= 4.0))
    return fail(h, MOP_ERR_ARG, "tuning factors out of range");
  h->tuning = *t;
  make_grid(h);
  drop_graph(h);
  for (auto& P : h->paths) {
    P.sized = false;     // strides and list shapes change: rebuild synchronously
    P.have_grad = false;
    P.list_ok = false;
  }
  return MOP_OK;
}

mop_status mop_set_list_skin(mop_handle* h, double skin_nm) {
  if (!h) return MOP_ERR_ARG;
  if (!std::isfinite(skin_nm) || skin_nm < 0.0) return fail(h, MOP_ERR_ARG, "skin must be finite and >= 0");
  const double half_box = 0.5 * std::min(h->box[0], std::min(h->box[1], h->box[2]));
  if (skin_nm > 0.0 && h->sc.rc + skin_nm >= half_box) return fail(h, MOP_ERR_ARG, "rc + skin must stay below L/2");
  h->skin = skin_nm;
  for (auto& P : h->paths) P.list_ok = false;
  return MOP_OK;
}

mop_status mop_get_list_stats(const mop_handle* h, int32_t path_id, int64_t* builds, int64_t* reuses) {
  if (!h || path_id < 0 || path_id >= kMaxPaths) return MOP_ERR_ARG;
  const PathHost& P = h->paths[path_id];
  if (!P.set) return MOP_ERR_STATE;
  if (builds) *builds = P.builds;
  if (reuses) *reuses = P.reuses;
  return MOP_OK;
}

mop_status mop_get_list_overflows(const mop_handle* h, int32_t path_id, int64_t* overflows) {
  if (!h || !overflows || path_id < 0 || path_id >= kMaxPaths) return MOP_ERR_ARG;
  const PathHost& P = h->paths[path_id];
  if (!P.set) return MOP_ERR_STATE;
  *overflows = P.overflows;
  return MOP_OK;
}

mop_status mop_get_tuning(const mop_handle* h, mop_tuning* t) {
  if (!h || !t) return MOP_ERR_ARG;
  *t = h->tuning;
  return MOP_OK;
}

mop_status mop_autotune(mop_handle* h, int32_t path_id, mop_tuning* best, double* best_ms) {
  if (!h) return MOP_ERR_ARG;
  std::vector<int> ids;
  mop_status s = select_paths(h, path_id, &ids);
  if (s) return s;
  CK(h, cudaSetDevice(h->device));
  cudaStream_t st = nullptr;
  cudaEvent_t e0, e1;
  CK(h, cudaEventCreate(&e0));
  CK(h, cudaEventCreate(&e1));
  const double cols[] = {0.85, 1.0, 1.2};
  const double bins[] = {0.5, 1.0};
  mop_tuning keep = h->tuning, win = h->tuning;
  double win_ms = 1e300;
  for (double c : cols)
    for (double b : bins) {
      const mop_tuning t{c, b};
      if ((s = mop_set_tuning(h, &t))) break;
      if ((s = evaluate(h, ids, nullptr, nullptr, st))) break;   // warm-up, sizes the lists
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && !s; ++r) s = evaluate(h, ids, nullptr, nullptr, st);
      cudaEventRecord(e1, st);
      if (s) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 2.0 < win_ms) {
        win_ms = ms / 2.0;
        win = t;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  mop_status s2 = mop_set_tuning(h, s ? &keep : &win);
  if (s) return s;
  if (s2) return s2;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return MOP_OK;
}

mop_status mop_metadynamics(mop_handle* h, int32_t n_deposits, int32_t stride, double dt_md, double gamma,
                            uint64_t seed, double height, double width, void* cuda_stream) {
  if (!h) return MOP_ERR_ARG;
  h->err.clear();
  if (n_deposits < 0 || stride < 1) return fail(h, MOP_ERR_ARG, "need n_deposits >= 0 and stride >= 1");
  if (!std::isfinite(height) || !std::isfinite(width) || !(width > 0))
    return fail(h, MOP_ERR_ARG, "invalid Gaussian height or width");
  std::vector<int> ids;
  mop_status s = select_paths(h, -1, &ids);
  if (s) return s;
  bool any = false;
  for (int id : ids) {
    const PathHost& P = h->paths[id];
    if (P.n_cv == 0) continue;
    any = true;
    if (P.n_gauss + n_deposits > kMaxGauss)
      return fail(h, MOP_ERR_ARG, "path %d would hold more than %d Gaussians", id, kMaxGauss);
  }
  if (!any) return fail(h, MOP_ERR_STATE, "no path has CV groups (mop_add_bias)");
  CK(h, cudaSetDevice(h->device));
  for (int id : ids) {
    PathHost& P = h->paths[id];
    if (P.n_cv == 0) continue;
    if ((s = ensure_gaussians(h, P))) return s;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  for (int d = 0; d < n_deposits; ++d) {
    if ((s = mop_step(h, stride, dt_md, gamma, seed, cuda_stream))) return s;
    // mop_step's last evaluation (eager or before the replays) left the table of all set paths,
    // with their current Gaussian counts, in d_paths; positions are current on the device
    Launch L{st, &h->launches};
    CK(h, launch_deposit(h->sc, h->d_paths.p, (int)ids.size(), height, width, L));
    for (int id : ids) {
      PathHost& P = h->paths[id];
      if (P.n_cv == 0) continue;
      ++P.n_gauss;
      P.have_grad = false;   // the next round starts from a gradient with the new Gaussian
    }
    CK(h, cudaStreamSynchronize(st));
  }
  return MOP_OK;
}

mop_status mop_get_gaussians(mop_handle* h, int32_t path_id, double* centers, double* heights, double* widths,
                             int32_t cap, int32_t* n, int32_t* n_cv) {
  if (!h) return MOP_ERR_ARG;
  h->err.clear();
  if (path_id < 0 || path_id >= kMaxPaths || cap < 0 || !n) return fail(h, MOP_ERR_ARG, "invalid argument");
  const PathHost& P = h->paths[path_id];
  *n = P.n_gauss;
  if (n_cv) *n_cv = P.n_cv;
  const int k = std::min(cap, P.n_gauss);
  if (k == 0) return MOP_OK;
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaDeviceSynchronize());
  const size_t row = sizeof(double) * kMaxCV, w = sizeof(double) * P.n_cv;
  if (centers) CK(h, cudaMemcpy2D(centers, w, P.gc.p, row, w, k, cudaMemcpyDeviceToHost));
  if (widths) CK(h, cudaMemcpy2D(widths, w, P.gw.p, row, w, k, cudaMemcpyDeviceToHost));
  if (heights) CK(h, cudaMemcpy(heights, P.gh.p, sizeof(double) * k, cudaMemcpyDeviceToHost));
  return MOP_OK;
}

mop_status mop_set_graph_mode(mop_handle* h, int32_t on) {
  if (!h) return MOP_ERR_ARG;
  h->graph_mode = on != 0;
  if (!h->graph_mode) drop_graph(h);
  return MOP_OK;
}

mop_status mop_kinetic_energy(mop_handle* h, int32_t path_id, double* ke) {
  if (!h) return MOP_ERR_ARG;
  if (!ke) return fail(h, MOP_ERR_ARG, "ke is NULL");
  std::vector<int> ids;
  mop_status s = select_paths(h, path_id, &ids);
  if (s || path_id < 0) return s ? s : fail(h, MOP_ERR_ARG, "path_id must be >= 0");
  CK(h, cudaSetDevice(h->device));
  PathHost& P = h->paths[path_id];
  if ((s = ensure_dynamics(h, ids, nullptr))) return s;
  CK(h, h->scratch.ensure(1));
  Launch L{nullptr, &h->launches};
  CK(h, launch_kinetic(h->sc, P.vel.p, P.N, h->scratch.p, L));
  CK(h, cudaMemcpy(ke, h->scratch.p, sizeof(double), cudaMemcpyDeviceToHost));
  return MOP_OK;
}

int32_t mop_last_launch_count(const mop_handle* h) { return h ? h->launches : 0; }

mop_status mop_set_profiling(mop_handle* h, int32_t on) {
  if (!h) return MOP_ERR_ARG;
  CK(h, cudaSetDevice(h->device));
  if (on && !h->ev[0])
    for (auto& e : h->ev) CK(h, cudaEventCreate(&e));
  h->profiling = on != 0;
  return MOP_OK;
}

mop_status mop_last_pass_ms(mop_handle* h, float* out, int32_t n) {
  if (!h) return MOP_ERR_ARG;
  if (!out || n < 0 || n > 6) return fail(h, MOP_ERR_ARG, "need 0 <= n <= 6 and an output array");
  if (!h->profiling) return fail(h, MOP_ERR_STATE, "profiling is off");
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaEventSynchronize(h->ev[6]));
  for (int k = 0; k < n; ++k) CK(h, cudaEventElapsedTime(&out[k], h->ev[k], h->ev[k + 1]));
  return MOP_OK;
}

mop_status mop_count_pairs(mop_handle* h, int32_t path_id, int64_t* unique, int64_t* listed) {
  if (!h) return MOP_ERR_ARG;
  if (!unique || !listed) return fail(h, MOP_ERR_ARG, "NULL output");
  int k = -1;
  for (size_t i = 0; i < h->last_ids.size(); ++i)
    if (h->last_ids[i] == path_id) k = (int)i;
  if (k < 0) return fail(h, MOP_ERR_STATE, "path %d was not in the last evaluation", path_id);
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaDeviceSynchronize());
  PathDev D = h->last_pd[k];
  D.unit_off = 0;
  CK(h, h->d_one.ensure(1));
  CK(h, h->counts.ensure(2));
  CK(h, cudaMemcpy(h->d_one.p, &D, sizeof(D), cudaMemcpyHostToDevice));
  int dummy = 0;
  Launch L{nullptr, &dummy};
  CK(h, launch_count_pairs(h->sc, h->d_one.p, 1, (long long)D.n_force * D.n_clu, h->counts.p, h->num_sms, L));
  (void)0;
  unsigned long long c[2];
  CK(h, cudaMemcpy(c, h->counts.p, sizeof(c), cudaMemcpyDeviceToHost));
  *unique = (int64_t)(c[0] / 2);
  *listed = (int64_t)c[1];
  return MOP_OK;
}

const char* mop_last_error(const mop_handle* h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
