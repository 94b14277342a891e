// C ABI of the bfmri library (include/bfmri.h): handle life cycle, state transfer, and the
// host-side orchestration of one Gibbs sweep (Section 3.2) as a fixed sequence of kernel
// launches on the handle's stream, with no host synchronisation inside a sweep.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/bfmri.h"
#include "model.cuh"
#include "mg.cuh"
#include "mrhs.cuh"
#include "pcg.cuh"
#include "summary.cuh"

using namespace bfmri;

namespace {
std::mutex g_err_mu;
std::string g_create_err = "no error";
}  // namespace

namespace bfmri {
// Process-wide error message (what bfmri_last_error(NULL) returns), for calls without a handle.
void set_global_error(const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_create_err = msg;
}
}  // namespace bfmri

namespace bfmri {
cudaError_t raise_smem_limit(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;   // (kernel, device) -> set limit
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{kern, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// Rows of the PCG partial-sum buffer of a handle: the largest streaming cooperative grid of
// its W (D = K) and A (D = P) solvers.
int handle_max_grid(int K, int P) {
  int maxgrid = pcg_max_grid(K);
  if (P > 0) maxgrid = std::max(maxgrid, pcg_max_grid(P));
  return maxgrid < 1 ? 1024 : maxgrid;
}

// Device bytes that bfmri_create allocates for a handle (each allocation rounded up to 256
// bytes as dalloc does), Y included: the peak of a request that runs create, statistics and
// Gibbs sweeps (no summaries, probes, grouped chains or SVB samples). Kept in step with
// bfmri_create's allocation list below.
size_t handle_device_bytes(int N, int T, int K, int P, size_t y_esz, bool mixed) {
  const size_t ld = ((size_t)N + 31) & ~size_t(31);
  const size_t D = std::max(K, P), Pa = std::max(P, 1);
  const size_t maxgrid = (size_t)handle_max_grid(K, P);
  auto r = [](size_t b) { return ((b == 0 ? 256 : b) + 255) & ~size_t(255); };
  size_t b = r(6 * ld * 4) + 3 * r(ld * 4) + r(ld) + r(4);                 // nbr, lin, red, black, colour, ctr
  b += r((size_t)T * N * y_esz) + r((size_t)T * K * 8);                    // Y, X
  b += r((size_t)n_stats(K, P) * ld * 8) + r((size_t)(P + 1) * (P + 1) * K * K * 8);
  b += r((size_t)K * ld * 8) + r(Pa * ld * 8) + r(ld * 8) + r((size_t)K * 8) + r(Pa * 8);
  b += r((size_t)n_syy(P) * ld * 8) + 2 * r((size_t)ntri((int)D) * ld * 8);
  b += 7 * r(D * ld * 8);                                                   // rhs, bmean, r, z, q, p0, p1
  b += r((maxgrid * 8 + 8) * 8) + r((size_t)hyper_grid(N) * D * 8);
  b += r(8) + r(4) + r(2 * sizeof(PcgCtrl)) + r(16);
  b += r(3 * D * ld * 8);                                                   // edge terms
  if (mixed) b += 2 * r((size_t)ntri((int)D) * ld * 4) + 6 * r(D * ld * 4);
  return b;
}

// Host geometry of the multigrid hierarchy of a lattice. Level l + 1 aggregates 2 x 2 x 2
// voxels of level l (2 x 2 in-slice for the 4-neighbour prior); there are at most
// MG_BUILD_LEVELS levels, and a coarsening is kept only while it shrinks the level and leaves
// at least 64 voxels. Each level holds its voxels in raster order of their coordinates and
// their neighbour slots; level 0's slot weights are the prior's per-direction weights, a
// coarse slot's weight is the sum of the weights of the fine edges joining the two aggregates
// (the Galerkin coarse graph of piecewise-constant prolongation).
constexpr int MG_BUILD_LEVELS = 3;

struct MgGeo {
  int N = 0, nx = 0, ny = 0, nz = 0;
  std::vector<int> x, y, z, nbr;   // nbr [6][N]: neighbour per slot (-x,+x,-y,+y,-z,+z) or -1
  std::vector<double> w;            // [6][N] slot weights (0 where there is no neighbour)
  std::vector<int> agg;             // [N] aggregate on the next level (all but the coarsest)
  std::vector<int> child;           // [8][N] voxels of the previous level (levels >= 1), -1 padding
  std::vector<int> red, black;      // voxels of even / odd coordinate sum
};

std::vector<MgGeo> mg_geometry(int nx, int ny, int nz, int ndir, const int* lin, int N, const double* cw) {
  const bool two_d = ndir == 4;
  std::vector<MgGeo> geo(1);
  geo.reserve(MG_BUILD_LEVELS);
  {
    MgGeo& g = geo[0];
    g.N = N;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    for (int n = 0; n < N; ++n) {
      g.x.push_back(lin[n] % nx);
      g.y.push_back((lin[n] / nx) % ny);
      g.z.push_back(lin[n] / (nx * ny));
    }
  }
  auto neighbours = [&](MgGeo& g) {
    std::vector<int> index((size_t)g.nx * g.ny * g.nz, -1);
    for (int n = 0; n < g.N; ++n) index[((size_t)g.z[n] * g.ny + g.y[n]) * g.nx + g.x[n]] = n;
    g.nbr.assign((size_t)6 * g.N, -1);
    g.w.assign((size_t)6 * g.N, 0.0);
    const int dx[6] = {-1, 1, 0, 0, 0, 0}, dy[6] = {0, 0, -1, 1, 0, 0}, dz[6] = {0, 0, 0, 0, -1, 1};
    for (int n = 0; n < g.N; ++n)
      for (int d = 0; d < ndir; ++d) {
        const int xx = g.x[n] + dx[d], yy = g.y[n] + dy[d], zz = g.z[n] + dz[d];
        if (xx < 0 || yy < 0 || zz < 0 || xx >= g.nx || yy >= g.ny || zz >= g.nz) continue;
        g.nbr[(size_t)d * g.N + n] = index[((size_t)zz * g.ny + yy) * g.nx + xx];
      }
    for (int n = 0; n < g.N; ++n) ((g.x[n] + g.y[n] + g.z[n]) & 1 ? g.black : g.red).push_back(n);
  };
  neighbours(geo[0]);
  for (int d = 0; d < 6; ++d)
    for (int n = 0; n < N; ++n)
      if (geo[0].nbr[(size_t)d * N + n] >= 0) geo[0].w[(size_t)d * N + n] = cw[d >> 1];
  while ((int)geo.size() < MG_BUILD_LEVELS) {
    MgGeo& f = geo.back();
    MgGeo c;
    c.nx = (f.nx + 1) / 2;
    c.ny = (f.ny + 1) / 2;
    c.nz = two_d ? f.nz : (f.nz + 1) / 2;
    std::vector<int> slot((size_t)c.nx * c.ny * c.nz, -1);
    auto cell = [&](int n) {
      return ((size_t)(two_d ? f.z[n] : f.z[n] / 2) * c.ny + f.y[n] / 2) * c.nx + f.x[n] / 2;
    };
    for (int n = 0; n < f.N; ++n) slot[cell(n)] = 0;
    for (size_t q = 0; q < slot.size(); ++q)
      if (slot[q] == 0) {
        slot[q] = c.N++;
        c.x.push_back((int)(q % c.nx));
        c.y.push_back((int)((q / c.nx) % c.ny));
        c.z.push_back((int)(q / ((size_t)c.nx * c.ny)));
      }
    if (c.N == f.N || c.N < 64) break;
    f.agg.assign(f.N, 0);
    c.child.assign((size_t)8 * c.N, -1);
    std::vector<int> cnt(c.N, 0);
    for (int n = 0; n < f.N; ++n) {
      const int a = slot[cell(n)];
      f.agg[n] = a;
      c.child[(size_t)(cnt[a]++) * c.N + a] = n;
    }
    neighbours(c);
    for (int n = 0; n < f.N; ++n)
      for (int d = 0; d < 6; ++d) {
        const int m = f.nbr[(size_t)d * f.N + n];
        if (m >= 0 && f.agg[n] != f.agg[m]) c.w[(size_t)d * c.N + f.agg[n]] += f.w[(size_t)d * f.N + n];
      }
    geo.push_back(std::move(c));   // capacity was reserved: f stays valid until here
  }
  return geo;
}

// Device bytes that ensure_mg allocates for a hierarchy (each allocation rounded up to 256
// bytes as dalloc does) for work planes of D components.
size_t mg_device_bytes(const std::vector<MgGeo>& geo, size_t ld0, int D) {
  auto r = [](size_t b) { return ((b == 0 ? 256 : b) + 255) & ~size_t(255); };
  const int L = (int)geo.size();
  size_t b = r(6 * ld0 * 8) + (L > 1 ? r(ld0 * 4) : 0);             // level 0: slot weights, aggregates
  for (int l = 1; l < L; ++l) {
    const size_t ld = ((size_t)geo[l].N + 31) & ~size_t(31);
    b += r(6 * ld * 4) + r(6 * ld * 8) + r(8 * ld * 4) + (l + 1 < L ? r(ld * 4) : 0);
    b += r(ld) + r(geo[l].red.size() * 4) + r(geo[l].black.size() * 4);
    b += 2 * r((size_t)ntri(D) * ld * 8) + 3 * r((size_t)D * ld * 8);
  }
  return b;
}

// The multigrid bytes of a request on a masked lattice (serving admission).
size_t mg_request_bytes(const bfmri_lattice& lat, const uint8_t* mask, int D) {
  std::vector<int> lin;
  const long long nsite = (long long)lat.nx * lat.ny * lat.nz;
  for (long long l = 0; l < nsite; ++l)
    if (mask[l]) lin.push_back((int)l);
  const double ones[3] = {1.0, 1.0, 1.0};
  const auto geo = mg_geometry(lat.nx, lat.ny, lat.nz, lat.neighbourhood, lin.data(), (int)lin.size(), ones);
  return mg_device_bytes(geo, ((size_t)lin.size() + 31) & ~size_t(31), D);
}
}  // namespace bfmri

struct bfmri_handle {
  int nx = 0, ny = 0, nz = 0, nbh = 6, ndir = 6;
  int N = 0, T = 0, K = 0, P = 0, D = 0;
  size_t ld = 0;
  bfmri_options opt{};
  cudaStream_t stream = nullptr;
  std::string err = "no error";
  std::vector<void*> allocs;
  std::vector<size_t> alloc_sizes;    // bytes of allocs[i] as requested from the allocator
  size_t bytes_now = 0, bytes_peak = 0;
  int* d_nbr = nullptr;
  int* d_lin = nullptr;
  void* d_Y = nullptr;
  int y_f64 = 1;
  double* d_X = nullptr;
  double* d_stats = nullptr;
  double* d_Sxx = nullptr;
  double *d_W = nullptr, *d_A = nullptr, *d_lam = nullptr, *d_alpha = nullptr, *d_beta = nullptr;
  double* d_G = nullptr;
  double *d_blocks = nullptr, *d_mfac = nullptr, *d_rhs = nullptr, *d_bmean = nullptr;
  double *d_r = nullptr, *d_z = nullptr, *d_q = nullptr, *d_p0 = nullptr, *d_p1 = nullptr;
  double *d_part = nullptr, *d_hpart = nullptr;
  // mixed precision (FP32 inner solver)
  float *d_blocks32 = nullptr, *d_mfac32 = nullptr, *d_u32 = nullptr, *d_r32 = nullptr;
  float *d_w32 = nullptr, *d_p32 = nullptr, *d_s32 = nullptr, *d_d32 = nullptr;
  double* d_edge = nullptr;   // [3][D][ld] perturbation edge terms
  unsigned int* d_bar = nullptr;
  int* d_err = nullptr;
  PcgCtrl* d_ctrl = nullptr;  // [0] W solves, [1] A solves, [2] auxiliary solves (exchange step)
  int* d_flags = nullptr;     // [0] bad voxel (min index), [1] Gamma draws out of attempts
  bool stats_ready = false;
  int part_rows = 0;
  std::vector<double> Sxx;
  std::vector<double> X_host;   // T x K design (digits of the tensor-core statistics)
  std::vector<int> lin_host;    // lattice-linear index of every voxel (multigrid hierarchy)
  std::vector<unsigned char> colour_host;   // 0 red, 1 black per voxel
  std::map<int, int> pair_slots;            // voxels per CTA -> lane pairs of k_pcg_rbp2
  double* d_ldm = nullptr;                  // log det M of a probe set riding with a group sweep
  double* d_lt = nullptr;                   // [K][ld] L v of the L'L prior's products
  unsigned short* d_ce = nullptr;           // [3][ld] BF16 per-edge factors of C, or null
  // anisotropic prior: alpha_{d,k} and the exchange step's proposal ([3][K] each), the
  // auxiliary field [K][ld], direction edge sums of W and of the field [2][3][K], log a [K]
  // and accepted steps [K]
  double *d_alpha3 = nullptr, *d_prop3 = nullptr, *d_waux = nullptr, *d_qdir = nullptr, *d_loga = nullptr;
  double* d_alam = nullptr;                 // [K] lam of the last ray move
  long long* d_acc = nullptr;
  int aniso_parts = 1;                      // connected parts of the voxel graph
  // multigrid hierarchy (BFMRI_PRECOND_MULTIGRID), built on the first multigrid solve:
  // levels 1..mg_L-1 plus level 0's slot weights and aggregate map
  int mg_L = 0;
  MgLevel mg_lv[MG_MAX_LEVELS];
  double* mg_wgt0 = nullptr;
  int* mg_agg0 = nullptr;
  int probe_tile = 1;           // right-hand-side tile of the last probe solve
  double probe_tile_ms[3] = {-1.0, -1.0, -1.0};   // autotuner's solve times of tiles 1, 2, 4

  int stride[3] = {1, 1, 1};
  int* d_red = nullptr;     // compact indices of the voxels with x + y + z even
  int* d_black = nullptr;   // and of the others (red-black SSOR phases)
  int n_red = 0, n_black = 0;
  unsigned char* d_colour = nullptr;   // [ld] 0 red, 1 black
  uint64_t mask_hash = 0;     // identity of the mask (FNV-1a of the in-mask lattice indices)
  // captured Gibbs sweep (options.use_graph): one sweep whose draws read the device counter
  uint32_t* d_sweep_ctr = nullptr;
  cudaGraph_t sweep_graph = nullptr;
  cudaGraphExec_t sweep_exec = nullptr;
  cudaStream_t capture_stream = nullptr;   // capture cannot run on the legacy default stream
  bool capturing = false;
  bool graph_failed = false;
  uint64_t uid = 0;                 // distinct for every handle the process creates
  // captured group sweep (this handle first in the group): the chains' uids and the
  // workspace it was captured with
  std::vector<uint64_t> gsweep_uids;
  const void* gsweep_ws = nullptr;
  cudaGraph_t gsweep_graph = nullptr;
  cudaGraphExec_t gsweep_exec = nullptr;
  bool gsweep_failed = false;
  // asynchronous sweeps (bfmri_gibbs_sweep without info) left their error words and PCG
  // counters unread: they accumulate until the next synchronising call
  bool deferred = false;
  // posterior summaries of the chain (bfmri_summary_begin .. bfmri_summary_end)
  struct Summary {
    bool open = false;
    int nc = 0;
    long long n = 0;
    bool has_set = false;
    double *ref = nullptr, *S1 = nullptr, *S2 = nullptr, *C = nullptr, *gamma = nullptr;
    double *mean = nullptr, *cov = nullptr, *ppm = nullptr;   // bfmri_summary_get output planes
    int* count = nullptr;
    uint8_t* in_set = nullptr;
    unsigned long long* joint = nullptr;
    unsigned int* scratch = nullptr;   // [2] joint-set failure word and CTA ticket
  } sum;
  double* d_lj = nullptr;   // log joint: [7] terms, [K] Q of W, [P] Q of A, CTA partials
  // grouped chains: per-chain operator tables [2][cap] and tallies [2][cap]
  MrhsRhsPtrs* d_gtab = nullptr;
  MrhsTally* d_gtally = nullptr;
  int g_cap = 0;
  // multi-right-hand-side workspace, grown on demand
  int mr_S = 0, mr_D = 0, mr_hist_len = 0, mr_units = 0;
  size_t mr_vs = 0;
  double *mr_b = nullptr, *mr_x = nullptr, *mr_r = nullptr, *mr_u = nullptr, *mr_w = nullptr;
  double *mr_p = nullptr, *mr_s = nullptr, *mr_part = nullptr, *mr_hist = nullptr, *mr_out = nullptr;
  size_t mr_out_len = 0;
  RhsState* mr_st = nullptr;
  int* mr_flags = nullptr;
  // spatial VB state: N_s samples of W and A (warm starts), work planes, extrapolation history
  int svb_S = 0, svb_iter = 0;
  double *svb_W = nullptr, *svb_A = nullptr, *svb_cmom = nullptr, *svb_gin = nullptr;
  double *svb_ldata = nullptr, *svb_part = nullptr, *d_zero = nullptr;
  std::vector<double> svb_alpha_hist[2], svb_beta_hist[2];
  // profiling: events recorded around launches, resolved lazily
  struct Pending { int cls; cudaEvent_t e0, e1; bool pcg; int which; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  bfmri_timing timing{};
};

namespace {

bfmri_status fail(bfmri_handle* h, bfmri_status code, const std::string& msg) {
  if (h) {
    h->err = msg;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_err = msg;
  }
  return code;
}

bfmri_status cuda_fail(bfmri_handle* h, cudaError_t e, const char* where) {
  return fail(h, BFMRI_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RET(x)                          \
  do {                                  \
    bfmri_status s_ = (x);              \
    if (s_ != BFMRI_OK) return s_;      \
  } while (0)

#define CU(h, call)                                    \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

void* dalloc(bfmri_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->opt.dev_alloc) {
    p = h->opt.dev_alloc(bytes, h->opt.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) {
    h->allocs.push_back(p);
    h->alloc_sizes.push_back(bytes);
    h->bytes_now += bytes;
    h->bytes_peak = std::max(h->bytes_peak, h->bytes_now);
  }
  return p;
}

void dfree(bfmri_handle* h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i) {
    if (h->allocs[i] == p) {
      h->bytes_now -= h->alloc_sizes[i];
      h->allocs.erase(h->allocs.begin() + i);
      h->alloc_sizes.erase(h->alloc_sizes.begin() + i);
      break;
    }
  }
  if (h->opt.dev_alloc) {
    if (h->opt.dev_free) h->opt.dev_free(p, h->opt.alloc_ctx);
  } else {
    cudaFree(p);
  }
}

// --- profiling -------------------------------------------------------------------------
cudaEvent_t take_event(bfmri_handle* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bfmri_status resolve_timing(bfmri_handle* h);

struct Timed {
  bfmri_handle* h;
  int cls;
  cudaEvent_t e0 = nullptr;
  bool pcg;
  int which;
  Timed(bfmri_handle* h_, int cls_, bool pcg_ = false, int which_ = 0) : h(h_), cls(cls_), pcg(pcg_), which(which_) {
    // profile 1: every launch; profile 2: the single-solve PCG launches only
    if (h->opt.profile == 1 || (h->opt.profile == 2 && pcg)) {
      if (h->pending.size() > 2048) resolve_timing(h);
      e0 = take_event(h);
      cudaEventRecord(e0, h->stream);
    }
  }
  ~Timed() {
    if (e0) {
      cudaEvent_t e1 = take_event(h);
      cudaEventRecord(e1, h->stream);
      h->pending.push_back({cls, e0, e1, pcg, which});
    }
  }
};

Geometry geom(const bfmri_handle* h) {
  Geometry g;
  g.N = h->N;
  g.ld = h->ld;
  g.ndir = h->ndir;
  g.nbr = h->d_nbr;
  g.lin = h->d_lin;
  g.stride[0] = h->stride[0];
  g.stride[1] = h->stride[1];
  g.stride[2] = h->stride[2];
  for (int d = 0; d < 3; ++d) g.cw[d] = h->opt.edge_weight[d];
  g.ce = h->d_ce;
  return g;
}

Rng rng_of(const bfmri_handle* h, uint64_t counter, uint32_t tag) {
  Rng r;
  r.k0 = (uint32_t)(h->opt.seed & 0xFFFFFFFFull);
  r.k1 = (uint32_t)(h->opt.seed >> 32);
  r.counter = (uint32_t)counter;
  r.c3 = (tag << 24) | (h->opt.stream_id & 0xFFFFFFu);
  r.dctr = nullptr;
  if (h->capturing) {   // the captured sweep reads its draw counter from the device word
    r.counter = 0u;
    r.dctr = h->d_sweep_ctr;
  }
  return r;
}

// host (rows x N row-major) <-> device planes (rows x ld)
bfmri_status to_dev(bfmri_handle* h, double* d, const double* src, int rows) {
  if (rows == 0) return BFMRI_OK;
  CU(h, cudaMemcpy2DAsync(d, h->ld * sizeof(double), src, (size_t)h->N * sizeof(double),
                          (size_t)h->N * sizeof(double), rows, cudaMemcpyHostToDevice, h->stream));
  return BFMRI_OK;
}

bfmri_status to_host(bfmri_handle* h, double* dst, const double* d, int rows) {
  if (rows == 0) return BFMRI_OK;
  CU(h, cudaMemcpy2DAsync(dst, (size_t)h->N * sizeof(double), d, h->ld * sizeof(double),
                          (size_t)h->N * sizeof(double), rows, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return BFMRI_OK;
}

bool all_finite(const double* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// Whether n FP64 (f64) or FP32 values are all finite, before any device work: a value is
// NaN or infinite exactly when its exponent bits are all set. The test runs without branches
// over blocks of values (so the compiler can vectorise it) on up to 8 host threads for large
// arrays, so a whole-brain series (about 120 MB) is checked in a few milliseconds.
bool values_finite(const void* v, size_t n, bool f64) {
  auto block_ok = [&](size_t i0, size_t i1) -> bool {
    if (f64) {
      const uint64_t* p = static_cast<const uint64_t*>(v);
      const uint64_t m = 0x7ff0000000000000ull;
      for (size_t b = i0; b < i1; b += 4096) {
        uint64_t bad = 0;
        const size_t e = std::min(i1, b + 4096);
        for (size_t i = b; i < e; ++i) bad |= (uint64_t)((p[i] & m) == m);
        if (bad) return false;
      }
    } else {
      const uint32_t* p = static_cast<const uint32_t*>(v);
      const uint32_t m = 0x7f800000u;
      for (size_t b = i0; b < i1; b += 4096) {
        uint32_t bad = 0;
        const size_t e = std::min(i1, b + 4096);
        for (size_t i = b; i < e; ++i) bad |= (uint32_t)((p[i] & m) == m);
        if (bad) return false;
      }
    }
    return true;
  };
  const size_t per = (size_t)1 << 22;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::min<size_t>({(size_t)8, (size_t)hw, (n + per - 1) / per});
  if (nt <= 1) return block_ok(0, n);
  std::vector<int> ok(nt, 1);
  std::vector<std::thread> th;
  const size_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] { ok[t] = block_ok(std::min(n, t * chunk), std::min(n, (t + 1) * chunk)) ? 1 : 0; });
  for (auto& x : th) x.join();
  for (int t = 0; t < nt; ++t)
    if (!ok[t]) return false;
  return true;
}

bool all_positive(const double* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!(v[i] > 0.0) || !std::isfinite(v[i])) return false;
  return true;
}

// Solvers that run the SSOR colour phases: SSOR itself, and the reduced red-black system
// wherever its own solver does not apply (there it is SSOR with omega = 1).
bool uses_ssor(const bfmri_options& o) {
  return o.precond == BFMRI_PRECOND_SSOR || o.precond == BFMRI_PRECOND_RB_REDUCED;
}
double ssor_omega_of(const bfmri_options& o) {
  return o.precond == BFMRI_PRECOND_RB_REDUCED ? 1.0 : o.ssor_omega;
}

// Clears the sticky device error words before a group of launches (kept, and added to,
// while the errors of asynchronous sweeps are unread).
bfmri_status begin_call(bfmri_handle* h) {
  if (h->deferred) return BFMRI_OK;
  CU(h, cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned int), h->stream));
  CU(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  CU(h, cudaMemsetAsync(h->d_ctrl, 0, 3 * sizeof(PcgCtrl), h->stream));
  CU(h, cudaMemsetAsync(h->d_flags, 0x7f, sizeof(int), h->stream));
  CU(h, cudaMemsetAsync(h->d_flags + 1, 0, 3 * sizeof(int), h->stream));
  return BFMRI_OK;
}

// Reads the device error words after synchronising; maps them to a status.
bfmri_status end_call(bfmri_handle* h, PcgCtrl* ctrl_out /* [2] or null */, int* exhausted) {
  h->deferred = false;
  CU(h, cudaStreamSynchronize(h->stream));
  PcgCtrl ctrl[3];
  int flags[4], err = 0;
  CU(h, cudaMemcpy(ctrl, h->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost));
  CU(h, cudaMemcpy(flags, h->d_flags, sizeof(flags), cudaMemcpyDeviceToHost));
  CU(h, cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (ctrl_out) {
    ctrl_out[0] = ctrl[0];
    ctrl_out[1] = ctrl[1];
  }
  if (h->opt.profile) {
    h->timing.pcg_iterations[BFMRI_T_PCG_W] += ctrl[0].iter_total;
    h->timing.pcg_iterations[BFMRI_T_PCG_A] += ctrl[1].iter_total;
    h->timing.pcg_iterations[BFMRI_T_HYPER] += ctrl[2].iter_total;
  }
  if (exhausted) *exhausted = flags[1];
  if (err == ERR_TIMEOUT_CODE)
    return fail(h, BFMRI_ERR_TIMEOUT, "device grid barrier wait exceeded its time limit");
  if (err == ERR_LAYOUT_CODE)
    return fail(h, BFMRI_ERR_INTERNAL, "solver launch layout does not match the voxel colours");
  if (flags[0] != 0x7f7f7f7f)
    return fail(h, BFMRI_ERR_NOT_SPD,
                "per-voxel block not positive definite at voxel " + std::to_string(flags[0]));
  for (int i = 0; i < 3; ++i) {
    const int st = ctrl[i].status_any;
    if (st == 4) return fail(h, BFMRI_ERR_NOT_CONVERGED, "PCG reached max_iter");
    if (st == 3) return fail(h, BFMRI_ERR_NOT_SPD, "PCG breakdown (p'Bp <= 0)");
    if (st == 7) return fail(h, BFMRI_ERR_INVALID_ARG, "non-finite value in PCG");
  }
  return BFMRI_OK;
}

// Multigrid hierarchy of the handle's lattice on the device (mg_geometry): per level its
// neighbour slots and weights, the children of every voxel, its aggregates on the next level,
// its colour lists, and blocks, factor and work planes for D = max(K, P). Level 0 uses the
// handle's own planes, lists, blocks and factor.
bfmri_status ensure_mg(bfmri_handle* h) {
  if (h->mg_L > 0) return BFMRI_OK;
  const int Dm = h->D;
  const std::vector<MgGeo> geo =
      mg_geometry(h->nx, h->ny, h->nz, h->ndir, h->lin_host.data(), h->N, h->opt.edge_weight);
  const int L = (int)geo.size();
  auto dcopy = [&](const void* src, size_t bytes) -> void* {
    void* p = dalloc(h, bytes);
    if (p && bytes && cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return nullptr;
    return p;
  };
  // planes [rows][ld] from host [rows][N]
  auto planes_i = [&](const std::vector<int>& v, int rows, int N, size_t ld) -> int* {
    std::vector<int> pad((size_t)rows * ld, -1);
    for (int r = 0; r < rows; ++r) std::copy(v.begin() + (size_t)r * N, v.begin() + (size_t)(r + 1) * N, pad.begin() + (size_t)r * ld);
    return (int*)dcopy(pad.data(), pad.size() * sizeof(int));
  };
  auto planes_d = [&](const std::vector<double>& v, int rows, int N, size_t ld) -> double* {
    std::vector<double> pad((size_t)rows * ld, 0.0);
    for (int r = 0; r < rows; ++r) std::copy(v.begin() + (size_t)r * N, v.begin() + (size_t)(r + 1) * N, pad.begin() + (size_t)r * ld);
    return (double*)dcopy(pad.data(), pad.size() * sizeof(double));
  };
  h->mg_wgt0 = planes_d(geo[0].w, 6, geo[0].N, h->ld);
  if (L > 1) h->mg_agg0 = planes_i(geo[0].agg, 1, geo[0].N, h->ld);
  if (!h->mg_wgt0 || (L > 1 && !h->mg_agg0)) return fail(h, BFMRI_ERR_OOM, "multigrid allocation failed");
  for (int l = 1; l < L; ++l) {
    const MgGeo& g = geo[l];
    MgLevel& v = h->mg_lv[l];
    memset(&v, 0, sizeof(v));
    v.N = g.N;
    v.ld = ((size_t)g.N + 31) & ~size_t(31);
    v.nbr = planes_i(g.nbr, 6, g.N, v.ld);
    v.wgt = planes_d(g.w, 6, g.N, v.ld);
    v.child = planes_i(g.child, 8, g.N, v.ld);
    if (l + 1 < L) v.agg = planes_i(g.agg, 1, g.N, v.ld);
    std::vector<unsigned char> col(v.ld, 0);
    for (int n : g.black) col[n] = 1;
    v.colour = (const unsigned char*)dcopy(col.data(), col.size());
    v.red = (const int*)dcopy(g.red.data(), g.red.size() * sizeof(int));
    v.black = (const int*)dcopy(g.black.data(), g.black.size() * sizeof(int));
    v.n_red = (int)g.red.size();
    v.n_black = (int)g.black.size();
    v.blocks = (const double*)dalloc(h, (size_t)ntri(Dm) * v.ld * sizeof(double));
    v.fac = (double*)dalloc(h, (size_t)ntri(Dm) * v.ld * sizeof(double));
    v.b = (double*)dalloc(h, (size_t)Dm * v.ld * sizeof(double));
    v.x = (double*)dalloc(h, (size_t)Dm * v.ld * sizeof(double));
    v.r = (double*)dalloc(h, (size_t)Dm * v.ld * sizeof(double));
    if (!v.nbr || !v.wgt || !v.child || (l + 1 < L && !v.agg) || !v.colour || !v.red || !v.black ||
        !v.blocks || !v.fac || !v.b || !v.x || !v.r)
      return fail(h, BFMRI_ERR_OOM, "multigrid allocation failed");
  }
  CU(h, cudaStreamSynchronize(h->stream));   // the host staging vectors go out of scope
  h->mg_L = L;
  return BFMRI_OK;
}

// Arguments of a multigrid solve of the system currently assembled in d_blocks / d_mfac
// (level 0's Gauss-Seidel factor is the block-Jacobi factor of blocks + diag(scale) deg).
MgArgs mg_args(bfmri_handle* h, const double* scale, double* x, int which) {
  MgArgs m;
  memset(&m, 0, sizeof(m));
  m.L = h->mg_L;
  m.coarse_steps = 2;
  MgLevel& z = m.lv[0];
  z.N = h->N;
  z.ld = h->ld;
  z.nbr = h->d_nbr;
  z.wgt = h->mg_wgt0;
  z.agg = h->mg_agg0;
  z.colour = h->d_colour;
  z.red = h->d_red;
  z.n_red = h->n_red;
  z.black = h->d_black;
  z.n_black = h->n_black;
  z.blocks = h->d_blocks;
  z.fac = h->d_mfac;
  z.b = h->d_r;
  z.x = h->d_z;
  z.r = h->d_p1;
  for (int l = 1; l < h->mg_L; ++l) m.lv[l] = h->mg_lv[l];
  m.scale = scale;
  m.b = h->d_rhs;
  m.x = x;
  m.r = h->d_r;
  m.z = h->d_z;
  m.p = h->d_p0;
  m.q = h->d_q;
  m.part = h->d_part;
  m.part1 = h->d_part + (size_t)h->part_rows * 4;
  m.max_grid = h->part_rows;
  m.sm_cap = h->opt.sm_budget;
  m.bar.count = h->d_bar;
  m.bar.gen = h->d_bar + 1;
  m.bar.err = h->d_err;
  m.bar.timeout_ns = (unsigned long long)(h->opt.barrier_timeout_s * 1e9);
  m.ctrl = h->d_ctrl + which;
  m.delta = h->opt.delta;
  m.max_iter = h->opt.max_iter;
  m.bad_voxel = h->d_flags;
  return m;
}

bfmri_status run_pcg_mg(bfmri_handle* h, int D, const double* scale, double* x, int which) {
  RET(ensure_mg(h));
  MgArgs m = mg_args(h, scale, x, which);
  Timed tm(h, which == 0 ? BFMRI_T_PCG_W : BFMRI_T_PCG_A, true, which);
  cudaError_t e = launch_mg_setup(D, m, h->stream);
  int grid = 0;
  if (e == cudaSuccess) e = launch_pcg_mg(D, m, h->stream, &grid);
  if (e != cudaSuccess) return cuda_fail(h, e, "multigrid PCG");
  return BFMRI_OK;
}

bfmri_status run_pcg(bfmri_handle* h, int D, const double* scale, double* x, int which) {
  if (h->opt.precond == BFMRI_PRECOND_MULTIGRID) return run_pcg_mg(h, D, scale, x, which);
  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.N = h->N;
  a.ld = h->ld;
  a.ndir = h->ndir;
  for (int d = 0; d < 3; ++d) a.cw[d] = h->opt.edge_weight[d];
  a.nbr = h->d_nbr;
  a.blocks = h->d_blocks;
  a.mfac = h->opt.precond != BFMRI_PRECOND_NONE ? h->d_mfac : nullptr;
  a.scale = scale;
  a.b = h->d_rhs;
  a.x = x;
  a.r = h->d_r;
  a.u = h->d_z;
  a.w = h->d_q;
  a.p = h->d_p0;
  a.s = h->d_p1;
  a.part = h->d_part;
  a.part1 = h->d_part + (size_t)h->part_rows * 4;
  a.allow_resident = h->opt.pcg_variant == BFMRI_PCG_AUTO;
  a.sm_cap = h->opt.sm_budget;
  a.mixed = h->opt.precision == BFMRI_PREC_MIXED;
  a.blocks32 = h->d_blocks32;
  a.mfac32 = h->opt.precond != BFMRI_PRECOND_NONE ? h->d_mfac32 : nullptr;
  a.ssor = uses_ssor(h->opt);
  a.omega = ssor_omega_of(h->opt);
  a.reduced = h->opt.precond == BFMRI_PRECOND_RB_REDUCED;
  if (which == 0 && h->opt.w_prior == BFMRI_PRIOR_LTL) {
    a.ltl = 1;
    a.t = h->d_lt;   // the block-Jacobi resident kernel where the voxels fit, else k_pcg_ltl
  }
  if (h->d_ce) a.ce = h->d_ce;   // block-Jacobi or reduced resident kernels, else streaming
  if (h->opt.w_prior == BFMRI_PRIOR_ANISO && which != 1) {
    // the W system (alpha_{d,k}) or the exchange step's auxiliary system (the proposal):
    // the block-Jacobi resident kernel where the voxels fit, else the streaming one
    a.scale3 = which == 0 ? h->d_alpha3 : h->d_prop3;
  }
  // lane pairs by default only for 6 x 6 blocks: measured on the whole-brain workload they
  // take the W solve (K = 6) from 0.414 to 0.404 ms per sweep, but the A solve (P = 3) from
  // 0.364 to 0.432 ms, where the second lane holds one component and the gathers and padded
  // triangular rows cost more than the extra warps save
  a.lanes = (h->opt.pcg_lanes == 2 || (h->opt.pcg_lanes == 0 && D >= 6)) ? 2 : 1;
  if (a.reduced && a.lanes == 2 && D <= 6) {
    // lane pairs of the resident solver: the most red, or black, voxels of any CTA
    const int per = resident_voxels_per_cta(h->N, h->opt.sm_budget);
    auto it = h->pair_slots.find(per);
    if (it == h->pair_slots.end()) {
      int slots = 0;
      for (int b0 = 0; b0 < h->N; b0 += per) {
        int nr = 0, nb = 0;
        for (int n = b0; n < std::min(h->N, b0 + per); ++n) (h->colour_host[n] ? nb : nr) += 1;
        slots = std::max(slots, std::max(nr, nb));
      }
      it = h->pair_slots.emplace(per, slots).first;
    }
    a.pair_per = per;
    a.pair_slots = it->second;
  }
  a.red = h->d_red;
  a.n_red = h->n_red;
  a.black = h->d_black;
  a.n_black = h->n_black;
  a.colour = h->d_colour;
  a.u32 = h->d_u32;
  a.r32 = h->d_r32;
  a.w32 = h->d_w32;
  a.p32 = h->d_p32;
  a.s32 = h->d_s32;
  a.d32 = h->d_d32;
  a.inner_tol = h->opt.inner_tol;
  a.max_inner = 1000;
  a.bar.count = h->d_bar;
  a.bar.gen = h->d_bar + 1;
  a.bar.err = h->d_err;
  a.bar.timeout_ns = (unsigned long long)(h->opt.barrier_timeout_s * 1e9);
  a.ctrl = h->d_ctrl + which;
  a.delta = h->opt.delta;
  a.max_iter = h->opt.max_iter;
  a.skip_block = h->opt.debug_skip_block;
  a.max_grid = h->part_rows;
  h->opt.debug_skip_block = -1;  // the hook fires once
  int grid = 0;
  Timed tm(h, which == 0 ? BFMRI_T_PCG_W : which == 1 ? BFMRI_T_PCG_A : BFMRI_T_HYPER, true, which);
  cudaError_t e = launch_pcg(D, a, h->stream, &grid);
  if (e != cudaSuccess) return cuda_fail(h, e, "launch_pcg");
  return BFMRI_OK;
}

AssembleArgs assemble_args(bfmri_handle* h, const double* scale, uint64_t counter, uint32_t tag) {
  AssembleArgs a;
  memset(&a, 0, sizeof(a));
  a.g = geom(h);
  a.K = h->K;
  a.P = h->P;
  a.stats = h->d_stats;
  a.Sxx = h->d_Sxx;
  a.W = h->d_W;
  a.A = h->d_A;
  a.lam = h->d_lam;
  a.scale = scale;
  a.eps = h->opt.eps;
  a.spatial = h->opt.ar_prior == BFMRI_AR_SPATIAL;
  a.perturb = 1;
  a.precond = h->opt.precond != BFMRI_PRECOND_NONE;
  a.rng = rng_of(h, counter, tag);
  a.blocks = h->d_blocks;
  a.mfac = h->d_mfac;
  a.blocks32 = h->d_blocks32;
  a.mfac32 = h->d_mfac32;
  a.rhs = h->d_rhs;
  a.G = h->d_G;
  a.bad_voxel = h->d_flags;
  a.ltl = tag == TAG_W && h->opt.w_prior == BFMRI_PRIOR_LTL;
  if (a.ltl) a.edge = h->d_edge;   // the prior terms, from launch_ltl_noise when perturbed
  if (tag == TAG_W && h->opt.w_prior == BFMRI_PRIOR_ANISO) a.scale3 = h->d_alpha3;
  return a;
}

// --- the five steps of a sweep, enqueued without synchronisation ---
// W system of the current state with perturbed right-hand side (Algorithm 2, steps 1-6).
bfmri_status assemble_W(bfmri_handle* h, uint64_t counter) {
  AssembleArgs a = assemble_args(h, h->d_alpha, counter, TAG_W);
  cudaError_t e;
  {
    Timed tm(h, BFMRI_T_ASSEMBLE_W);
    e = a.ltl ? launch_ltl_noise(a.g, h->K, h->d_alpha, a.rng, h->d_edge, h->stream)
              : launch_edge_noise(a.g, h->K, h->d_alpha, a.rng, h->d_edge, h->stream, a.scale3);
    a.edge = h->d_edge;
    if (e == cudaSuccess) e = launch_assemble_w(a, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble_w");
  return BFMRI_OK;
}

bfmri_status enqueue_W(bfmri_handle* h, uint64_t counter) {
  RET(assemble_W(h, counter));
  return run_pcg(h, h->K, h->d_alpha, h->d_W, 0);
}

// A system (spatial prior) or the per-voxel A draw (independent prior, or the lagged Gram
// alone when P = 0).
bfmri_status assemble_A(bfmri_handle* h, uint64_t counter) {
  AssembleArgs a = assemble_args(h, h->d_beta, counter, TAG_A);
  const bool spatial = h->opt.ar_prior == BFMRI_AR_SPATIAL;
  if (h->P == 0) {
    a.g_only = 1;
  } else if (!spatial) {
    a.rhs = nullptr;
    a.x_direct = h->d_A;
    a.precond = 0;
  }
  cudaError_t e = cudaSuccess;
  {
    Timed tm(h, BFMRI_T_ASSEMBLE_A);
    if (h->P > 0 && spatial) {
      e = launch_edge_noise(a.g, h->P, h->d_beta, a.rng, h->d_edge, h->stream);
      a.edge = h->d_edge;
    }
    if (e == cudaSuccess) e = launch_assemble_a(a, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble_a");
  return BFMRI_OK;
}

bfmri_status enqueue_A(bfmri_handle* h, uint64_t counter) {
  RET(assemble_A(h, counter));
  if (h->P > 0 && h->opt.ar_prior == BFMRI_AR_SPATIAL) return run_pcg(h, h->P, h->d_beta, h->d_A, 1);
  return BFMRI_OK;
}

bfmri_status enqueue_gram(bfmri_handle* h) {
  AssembleArgs a = assemble_args(h, h->d_beta, 0, TAG_A);
  a.g_only = 1;
  cudaError_t e = launch_assemble_a(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble_a(gram)");
  return BFMRI_OK;
}

bfmri_status enqueue_lambda(bfmri_handle* h, uint64_t counter) {
  LambdaArgs a;
  a.g = geom(h);
  a.P = h->P;
  a.T = h->T;
  a.u1 = h->opt.u1;
  a.u2 = h->opt.u2;
  a.G = h->d_G;
  a.A = h->d_A;
  a.lam = h->d_lam;
  a.rng = rng_of(h, counter, TAG_LAMBDA);
  a.exhausted = h->d_flags + 1;
  Timed tm(h, BFMRI_T_LAMBDA);
  cudaError_t e = launch_lambda(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "lambda");
  return BFMRI_OK;
}

// Adds the current W as one sample to the open chain summary (kernels_summary.cu).
bfmri_status enqueue_summary(bfmri_handle* h) {
  ChainSumArgs a;
  a.g = geom(h);
  a.K = h->K;
  a.nc = h->sum.nc;
  a.W = h->d_W;
  a.ref = h->sum.ref;
  a.C = h->sum.C;
  a.gamma = h->sum.gamma;
  a.in_set = h->sum.has_set ? h->sum.in_set : nullptr;
  a.S1 = h->sum.S1;
  a.S2 = h->sum.S2;
  a.count = h->sum.count;
  a.joint = h->sum.joint;
  a.fail = h->sum.scratch;
  a.ticket = h->sum.scratch + 1;
  Timed tm(h, BFMRI_T_SUMMARY);
  const cudaError_t e = launch_chain_accumulate(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "chain summary");
  return BFMRI_OK;
}

// Anisotropic prior: alpha_k as the mean of alpha_{d,k} over the lattice's directions.
bfmri_status alpha_dir_mean(bfmri_handle* h, double* alpha) {
  std::vector<double> a3(3 * (size_t)h->K);
  CU(h, cudaMemcpyAsync(a3.data(), h->d_alpha3, a3.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  const int nd = h->ndir / 2;
  for (int k = 0; k < h->K; ++k) {
    double m = 0.0;
    for (int d = 0; d < nd; ++d) m += a3[(size_t)d * h->K + k];
    alpha[k] = m / nd;
  }
  return BFMRI_OK;
}

// The anisotropic prior's alpha step for every k: the direction edge sums of W, the exact ray
// move alpha -> lam alpha, then one exchange step (proposal, auxiliary prior draw into d_waux
// through the W system's buffers, the field's edge sums, acceptance).
bfmri_status enqueue_aniso(bfmri_handle* h, uint64_t counter) {
  const int K = h->K;
  AnisoArgs s;
  s.K = K;
  s.nd = h->ndir / 2;
  s.step = h->opt.aniso_step > 0.0 ? h->opt.aniso_step : 1.0 / sqrt((double)h->N);
  s.q1 = h->opt.q1;
  s.q2 = h->opt.q2;
  s.alpha3 = h->d_alpha3;
  s.prop3 = h->d_prop3;
  s.Q = h->d_qdir;
  s.Qp = h->d_qdir + 3 * K;
  s.log_a = h->d_loga;
  s.accepted = h->d_acc;
  s.rng = rng_of(h, counter, TAG_ALPHA_PROP);
  s.N = h->N;
  s.parts = h->aniso_parts;
  s.lam = h->d_alam;
  s.rng_scale = rng_of(h, counter, TAG_ALPHA);
  s.exhausted = h->d_flags + 1;
  const Geometry g = geom(h);
  HyperArgs q;
  q.g = g;
  q.D = K;
  q.part = h->d_hpart;
  q.out = nullptr;
  q.rng = s.rng;
  q.exhausted = h->d_flags + 1;
  q.ltl = 0;
  q.dirs = 1;
  cudaError_t e;
  {
    Timed tm(h, BFMRI_T_HYPER);
    // direction edge sums of W, the ray move, then the exchange step's proposal
    q.V = h->d_W;
    q.Q_out = h->d_qdir;
    e = launch_hyper(q, h->stream);
    if (e == cudaSuccess) e = launch_aniso_scale(s, h->stream);
    if (e == cudaSuccess) e = launch_aniso_propose(s, h->stream);
    if (e == cudaSuccess)
      e = launch_edge_noise(g, K, h->d_alpha, rng_of(h, counter, TAG_ALPHA_AUX), h->d_edge, h->stream, h->d_prop3);
    if (e == cudaSuccess)
      e = launch_aux_system(g, K, h->d_prop3, h->d_edge, h->d_blocks, h->d_mfac, h->d_rhs, h->d_waux, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "exchange step (proposal)");
  RET(run_pcg(h, K, h->d_alpha, h->d_waux, 2));
  {
    Timed tm(h, BFMRI_T_HYPER);
    q.V = h->d_waux;
    q.Q_out = h->d_qdir + 3 * K;
    e = launch_hyper(q, h->stream);
    if (e == cudaSuccess) e = launch_aniso_accept(s, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "exchange step (acceptance)");
  return BFMRI_OK;
}

bfmri_status enqueue_hyper(bfmri_handle* h, uint64_t counter, bool beta) {
  if (!beta && h->opt.w_prior == BFMRI_PRIOR_ANISO) return enqueue_aniso(h, counter);
  HyperArgs a;
  a.g = geom(h);
  a.D = beta ? h->P : h->K;
  a.V = beta ? h->d_A : h->d_W;
  a.part = h->d_hpart;
  a.prior1 = beta ? h->opt.r1 : h->opt.q1;
  a.prior2 = beta ? h->opt.r2 : h->opt.q2;
  a.out = beta ? h->d_beta : h->d_alpha;
  a.Q_out = nullptr;
  a.rng = rng_of(h, counter, beta ? TAG_BETA : TAG_ALPHA);
  a.exhausted = h->d_flags + 1;
  a.ltl = !beta && h->opt.w_prior == BFMRI_PRIOR_LTL;
  Timed tm(h, BFMRI_T_HYPER);
  cudaError_t e = launch_hyper(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "hyper");
  return BFMRI_OK;
}

bfmri_status resolve_timing(bfmri_handle* h) {
  if (h->pending.empty()) return BFMRI_OK;
  CU(h, cudaStreamSynchronize(h->stream));
  for (auto& p : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      h->timing.ms[p.cls] += ms;
      h->timing.launches[p.cls] += 1;
    }
    h->event_pool.push_back(p.e0);
    h->event_pool.push_back(p.e1);
  }
  h->pending.clear();
  return BFMRI_OK;
}

// Multi-RHS buffers for S right-hand sides of dimension D and hist_len recorded iterations.
bfmri_status ensure_mrhs(bfmri_handle* h, int D, int S, int hist_len, size_t ld_max = 0, int N_max = 0) {
  // a group of chains on different lattices sizes the workspace for the largest of them
  const size_t ldw = std::max(h->ld, ld_max);
  const int Nw = std::max(h->N, N_max);
  const size_t vs = (size_t)D * ldw;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // rows of the partial buffer: one per (RHS, chunk) unit, never more than max(warps, S);
  // right-hand-side tiles of up to 4 multiply the rows per warp by the tile
  const int units = std::max(std::max(nsm, 1) * 64 * 4, S);
  const size_t out_len = std::max(ldw, (size_t)((Nw + 127) / 128 + 1) * S * D);
  if (S <= h->mr_S && D <= h->mr_D && hist_len <= h->mr_hist_len && units <= h->mr_units &&
      out_len <= h->mr_out_len && vs <= h->mr_vs)
    return BFMRI_OK;
  double** vecs[] = {&h->mr_b, &h->mr_x, &h->mr_r, &h->mr_u, &h->mr_w, &h->mr_p, &h->mr_s};
  for (double** v : vecs) {
    dfree(h, *v);
    *v = nullptr;
  }
  dfree(h, h->mr_part);
  dfree(h, h->mr_hist);
  dfree(h, h->mr_out);
  dfree(h, h->mr_st);
  dfree(h, h->mr_flags);
  h->mr_S = h->mr_D = h->mr_hist_len = h->mr_units = 0;
  h->mr_vs = 0;
  for (double** v : vecs) {
    *v = (double*)dalloc(h, (size_t)S * vs * sizeof(double));
    if (!*v) return fail(h, BFMRI_ERR_OOM, "multi-RHS workspace allocation failed");
  }
  h->mr_part = (double*)dalloc(h, (size_t)units * 4 * sizeof(double));
  h->mr_hist = (double*)dalloc(h, (size_t)std::max(hist_len, 1) * S * 2 * sizeof(double));
  h->mr_out = (double*)dalloc(h, out_len * sizeof(double));
  h->mr_st = (RhsState*)dalloc(h, (size_t)S * sizeof(RhsState));
  h->mr_flags = (int*)dalloc(h, 4 * sizeof(int));
  if (!h->mr_part || !h->mr_hist || !h->mr_out || !h->mr_st || !h->mr_flags)
    return fail(h, BFMRI_ERR_OOM, "multi-RHS workspace allocation failed");
  h->mr_S = S;
  h->mr_D = D;
  h->mr_vs = vs;
  h->mr_hist_len = hist_len;
  h->mr_units = units;
  h->mr_out_len = out_len;
  return BFMRI_OK;
}

MrhsArgs mrhs_args(bfmri_handle* h, int D, int S, const double* scale, int max_iter, bool hist) {
  MrhsArgs m;
  memset(&m, 0, sizeof(m));
  m.N = h->N;
  m.ld = h->ld;
  m.ndir = h->ndir;
  m.f32 = 0;
  m.nbr = h->d_nbr;
  m.blocks = h->d_blocks;
  m.mfac = h->opt.precond != BFMRI_PRECOND_NONE ? h->d_mfac : nullptr;   // block-Jacobi
  m.scale = scale;
  m.S = S;
  m.vs = h->mr_vs;
  m.b = h->mr_b;
  m.x = h->mr_x;
  m.r = h->mr_r;
  m.u = h->mr_u;
  m.w = h->mr_w;
  m.p = h->mr_p;
  m.s = h->mr_s;
  m.part = h->mr_part;
  m.st = h->mr_st;
  m.hist = hist ? h->mr_hist : nullptr;
  m.hist_len = hist ? h->mr_hist_len : 0;
  m.flags = h->mr_flags;
  m.bar.count = h->d_bar;
  m.bar.gen = h->d_bar + 1;
  m.bar.err = h->d_err;
  m.bar.timeout_ns = (unsigned long long)(h->opt.barrier_timeout_s * 1e9);
  m.delta = h->opt.delta;
  m.max_iter = max_iter;
  m.max_restarts = 4;
  m.sm_cap = h->opt.sm_budget;
  for (int d = 0; d < 3; ++d) m.cw[d] = h->opt.edge_weight[d];
  return m;
}

// Red-black SSOR, or CG on the red-black reduced system, for the plain multi-RHS solves (SVB
// samples, grouped chains) when the handle asks for it; the probe solves keep block-Jacobi.
void mrhs_ssor(const bfmri_handle* h, MrhsArgs& m) {
  m.reduced = h->opt.precond == BFMRI_PRECOND_RB_REDUCED;
  m.ssor = uses_ssor(h->opt) && !m.reduced;
  m.omega = ssor_omega_of(h->opt);
  m.red = h->d_red;
  m.n_red = h->n_red;
  m.black = h->d_black;
  m.n_black = h->n_black;
}

bfmri_status require_stats(bfmri_handle* h) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (!h->stats_ready) return fail(h, BFMRI_ERR_STATE, "bfmri_precompute_stats has not run");
  return BFMRI_OK;
}

void fill_info(bfmri_solve_info* info, const PcgCtrl& c) {
  if (!info) return;
  info->iterations = c.iterations;
  info->refinements = c.restarts;
  info->rel_residual = c.rel_res;
  info->rel_residual0 = c.rel_res0;
}

}  // namespace

extern "C" {

void bfmri_default_options(bfmri_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->q1 = 10.0;
  o->q2 = 0.1;
  o->u1 = 10.0;
  o->u2 = 0.1;
  o->r1 = 10000.0;
  o->r2 = 0.1;
  o->eps = 0.0;
  o->delta = 1e-8;
  o->max_iter = 2000;
  o->precond = BFMRI_PRECOND_BLOCK_JACOBI;
  o->ssor_omega = 1.0;
  o->use_graph = 0;
  o->edge_weight[0] = o->edge_weight[1] = o->edge_weight[2] = 1.0;
  o->precision = BFMRI_PREC_FP64;
  o->ar_prior = BFMRI_AR_SPATIAL;
  o->y_layout = BFMRI_Y_MASKED;
  o->inner_tol = 1e-6;
  o->seed = 0x5eed5eedULL;
  o->stream_id = 0;
  o->cuda_stream = nullptr;
  o->barrier_timeout_s = 2.0;
  o->debug_skip_block = -1;
  o->stats_kernel = BFMRI_STATS_AUTO;
  o->mrhs_tile = 0;
  o->w_prior = BFMRI_PRIOR_UGL;
  o->pcg_lanes = 0;
  o->aniso_step = 0.0;
}

const char* bfmri_last_error(const bfmri_handle* h) {
  if (h) return h->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  static thread_local std::string copy;
  copy = g_create_err;
  return copy.c_str();
}

int bfmri_num_voxels(const bfmri_handle* h) { return h ? h->N : 0; }

bfmri_status bfmri_probe_tuning(const bfmri_handle* h, int* tile, double* ms) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (tile) *tile = h->probe_tile;
  if (ms)
    for (int c = 0; c < 3; ++c) ms[c] = h->probe_tile_ms[c];
  return BFMRI_OK;
}

bfmri_status bfmri_device_bytes(const bfmri_handle* h, size_t* now, size_t* peak) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (now) *now = h->bytes_now;
  if (peak) *peak = h->bytes_peak;
  return BFMRI_OK;
}

bfmri_status bfmri_sizes(const bfmri_handle* h, int* N, int* T, int* K, int* P) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (N) *N = h->N;
  if (T) *T = h->T;
  if (K) *K = h->K;
  if (P) *P = h->P;
  return BFMRI_OK;
}

bfmri_status bfmri_create(const bfmri_lattice* lat, const uint8_t* mask, const double* X,
                          const void* Y, int y_dtype, int T, int K, int P,
                          const bfmri_options* opt, bfmri_handle** out) {
  if (!out) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!lat || !mask || !X || !Y) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "NULL input");
  if (lat->nx < 1 || lat->ny < 1 || lat->nz < 1)
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "lattice dimensions must be positive");
  if (lat->neighbourhood != 4 && lat->neighbourhood != 6)
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "neighbourhood must be 4 or 6");
  if (K < 1 || K > KMAX) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "K must be in [1, 12]");
  if (P < 0 || P > PMAX) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "P must be in [0, 4]");
  if (T <= P + K) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "T must exceed P + K");
  if (y_dtype != BFMRI_F32 && y_dtype != BFMRI_F64)
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "y_dtype must be BFMRI_F32 or BFMRI_F64");
  const long long nsite = (long long)lat->nx * lat->ny * lat->nz;
  if (nsite >= (1LL << 30)) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "lattice too large (>= 2^30 sites)");
  bfmri_options o;
  if (opt) o = *opt; else bfmri_default_options(&o);
  if (!(o.delta > 0.0) || o.max_iter < 1 || !(o.barrier_timeout_s > 0.0) || o.eps < 0.0 ||
      !(o.q1 > 0) || !(o.q2 > 0) || !(o.u1 > 0) || !(o.u2 > 0) || !(o.r1 > 0) || !(o.r2 > 0))
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "invalid option value");
  if (o.sm_budget < 0) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "sm_budget must be >= 0");
  if (o.pcg_variant != BFMRI_PCG_AUTO && o.pcg_variant != BFMRI_PCG_STREAMING)
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "unknown pcg_variant");
  if (o.precond != BFMRI_PRECOND_NONE && o.precond != BFMRI_PRECOND_BLOCK_JACOBI &&
      o.precond != BFMRI_PRECOND_SSOR && o.precond != BFMRI_PRECOND_RB_REDUCED &&
      o.precond != BFMRI_PRECOND_MULTIGRID)
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "unknown preconditioner");
  if (o.precond == BFMRI_PRECOND_SSOR && !(o.ssor_omega > 0.0 && o.ssor_omega < 2.0))
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "ssor_omega must be in (0, 2)");
  if (o.precision != BFMRI_PREC_FP64 && o.precision != BFMRI_PREC_MIXED)
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "unknown precision mode");
  for (int d = 0; d < 3; ++d)
    if (!(o.edge_weight[d] > 0.0) || !std::isfinite(o.edge_weight[d]))
      return fail(nullptr, BFMRI_ERR_INVALID_ARG, "edge_weight must be positive and finite");
  if (o.pcg_lanes < 0 || o.pcg_lanes > 2) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "pcg_lanes must be 0, 1 or 2");
  if (o.w_prior != BFMRI_PRIOR_UGL && o.w_prior != BFMRI_PRIOR_LTL && o.w_prior != BFMRI_PRIOR_ANISO)
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "unknown w_prior");
  if (o.w_prior == BFMRI_PRIOR_ANISO &&
      ((o.precond != BFMRI_PRECOND_NONE && o.precond != BFMRI_PRECOND_BLOCK_JACOBI &&
        o.precond != BFMRI_PRECOND_RB_REDUCED) ||
       o.precision != BFMRI_PREC_FP64 || !std::isfinite(o.aniso_step)))
    return fail(nullptr, BFMRI_ERR_INVALID_ARG,
                "the anisotropic prior needs the reduced red-black, block-Jacobi or no preconditioner, "
                "FP64 precision and a finite aniso_step");
  if (o.w_prior == BFMRI_PRIOR_LTL &&
      ((o.precond != BFMRI_PRECOND_NONE && o.precond != BFMRI_PRECOND_BLOCK_JACOBI) ||
       o.precision != BFMRI_PREC_FP64))
    return fail(nullptr, BFMRI_ERR_INVALID_ARG,
                "the L'L prior needs block-Jacobi or no preconditioner and FP64 precision");
  if (o.stats_kernel != BFMRI_STATS_AUTO && o.stats_kernel != BFMRI_STATS_FP64 &&
      o.stats_kernel != BFMRI_STATS_TENSOR)
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "unknown stats_kernel");
  if (o.precision == BFMRI_PREC_MIXED && !(o.inner_tol > 0.0 && o.inner_tol < 1.0))
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
  if (!all_finite(X, (size_t)T * K)) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "X has non-finite values");

  // in-mask voxels in raster order and their neighbour planes
  std::vector<int> index_of((size_t)nsite, -1), lin;
  for (long long l = 0; l < nsite; ++l)
    if (mask[l]) {
      index_of[(size_t)l] = (int)lin.size();
      lin.push_back((int)l);
    }
  const int N = (int)lin.size();
  if (N == 0) return fail(nullptr, BFMRI_ERR_INVALID_ARG, "mask is empty");

  bfmri_handle* h = new bfmri_handle();
  h->opt = o;
  {
    static std::atomic<uint64_t> next_uid{1};
    h->uid = next_uid.fetch_add(1);
  }
  h->mask_hash = 1469598103934665603ull;
  for (int l : lin) {
    for (int byte = 0; byte < 4; ++byte) {
      h->mask_hash ^= (uint64_t)(((unsigned)l >> (8 * byte)) & 0xFFu);
      h->mask_hash *= 1099511628211ull;
    }
  }
  h->nx = lat->nx;
  h->ny = lat->ny;
  h->nz = lat->nz;
  h->nbh = lat->neighbourhood;
  h->ndir = lat->neighbourhood;
  h->N = N;
  h->T = T;
  h->K = K;
  h->P = P;
  h->D = K > P ? K : P;
  h->ld = ((size_t)N + 31) & ~size_t(31);
  h->stream = (cudaStream_t)o.cuda_stream;
  h->stride[0] = 1;
  h->stride[1] = lat->nx;
  h->stride[2] = lat->nx * lat->ny;
  const size_t ld = h->ld;

  std::vector<int> nbr(6 * ld, -1);
  for (int n = 0; n < N; ++n) {
    const int l = lin[n];
    const int x = l % lat->nx, y = (l / lat->nx) % lat->ny, z = l / (lat->nx * lat->ny);
    const int dx[6] = {-1, 1, 0, 0, 0, 0}, dy[6] = {0, 0, -1, 1, 0, 0}, dz[6] = {0, 0, 0, 0, -1, 1};
    for (int d = 0; d < h->ndir; ++d) {
      const int xx = x + dx[d], yy = y + dy[d], zz = z + dz[d];
      if (xx < 0 || yy < 0 || zz < 0 || xx >= lat->nx || yy >= lat->ny || zz >= lat->nz) continue;
      nbr[d * ld + n] = index_of[(size_t)zz * lat->nx * lat->ny + (size_t)yy * lat->nx + xx];
    }
  }
  // Y restricted to the mask, validated
  const size_t ycols = o.y_layout == BFMRI_Y_LATTICE ? (size_t)nsite : (size_t)N;
  const size_t esz = y_dtype == BFMRI_F64 ? 8 : 4;
  std::vector<unsigned char> ymask;
  const void* ysrc = Y;
  if (o.y_layout == BFMRI_Y_LATTICE) {
    ymask.resize((size_t)T * N * esz);
    for (int t = 0; t < T; ++t)
      for (int n = 0; n < N; ++n)
        memcpy(&ymask[((size_t)t * N + n) * esz],
               static_cast<const unsigned char*>(Y) + ((size_t)t * ycols + lin[n]) * esz, esz);
    ysrc = ymask.data();
  }
  if (!values_finite(ysrc, (size_t)T * N, y_dtype == BFMRI_F64)) {
    delete h;
    return fail(nullptr, BFMRI_ERR_INVALID_ARG, "Y has non-finite values");
  }
  h->X_host.assign(X, X + (size_t)T * K);
  h->lin_host = lin;
  if (o.w_prior == BFMRI_PRIOR_ANISO) {
    // connected parts of the voxel graph (the ray move's pseudo-determinant exponent N - parts)
    std::vector<int> part(N, -1), stack;
    int parts = 0;
    for (int s0 = 0; s0 < N; ++s0) {
      if (part[s0] >= 0) continue;
      part[s0] = parts;
      stack.assign(1, s0);
      while (!stack.empty()) {
        const int n = stack.back();
        stack.pop_back();
        for (int d = 0; d < h->ndir; ++d) {
          const int m = nbr[(size_t)d * ld + n];
          if (m >= 0 && part[m] < 0) {
            part[m] = parts;
            stack.push_back(m);
          }
        }
      }
      ++parts;
    }
    h->aniso_parts = parts;
  }
  // voxel-independent lagged X products Sxx[p][q][i][j] over t = P+1..T (1-based)
  h->Sxx.assign((size_t)(P + 1) * (P + 1) * K * K, 0.0);
  for (int p = 0; p <= P; ++p)
    for (int q = 0; q <= P; ++q)
      for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
          double s = 0.0;
          for (int t = P; t < T; ++t) s += X[(t - p) + (size_t)T * i] * X[(t - q) + (size_t)T * j];
          h->Sxx[(((size_t)p * (P + 1) + q) * K + i) * K + j] = s;
        }

  // device memory
  auto A = [&](size_t bytes) { return dalloc(h, bytes); };
  const int D = h->D;
  const int Pa = P > 0 ? P : 1;
  const int maxgrid = handle_max_grid(K, P);
  h->part_rows = maxgrid;
  h->d_nbr = (int*)A(6 * ld * sizeof(int));
  h->d_lin = (int*)A(ld * sizeof(int));
  h->d_red = (int*)A(ld * sizeof(int));
  h->d_black = (int*)A(ld * sizeof(int));
  h->d_colour = (unsigned char*)A(ld);
  h->d_sweep_ctr = (uint32_t*)A(sizeof(uint32_t));
  h->d_Y = A((size_t)T * N * esz);
  h->y_f64 = y_dtype == BFMRI_F64;
  h->d_X = (double*)A((size_t)T * K * sizeof(double));
  h->d_stats = (double*)A((size_t)n_stats(K, P) * ld * sizeof(double));
  h->d_Sxx = (double*)A(h->Sxx.size() * sizeof(double));
  h->d_W = (double*)A((size_t)K * ld * sizeof(double));
  h->d_A = (double*)A((size_t)Pa * ld * sizeof(double));
  h->d_lam = (double*)A(ld * sizeof(double));
  h->d_alpha = (double*)A((size_t)K * sizeof(double));
  h->d_beta = (double*)A((size_t)Pa * sizeof(double));
  h->d_G = (double*)A((size_t)n_syy(P) * ld * sizeof(double));
  h->d_blocks = (double*)A((size_t)ntri(D) * ld * sizeof(double));
  h->d_mfac = (double*)A((size_t)ntri(D) * ld * sizeof(double));
  h->d_rhs = (double*)A((size_t)D * ld * sizeof(double));
  h->d_bmean = (double*)A((size_t)D * ld * sizeof(double));
  h->d_r = (double*)A((size_t)D * ld * sizeof(double));
  h->d_z = (double*)A((size_t)D * ld * sizeof(double));
  h->d_q = (double*)A((size_t)D * ld * sizeof(double));
  h->d_p0 = (double*)A((size_t)D * ld * sizeof(double));
  h->d_p1 = (double*)A((size_t)D * ld * sizeof(double));
  h->d_part = (double*)A(((size_t)maxgrid * 8 + 8) * sizeof(double));
  // the anisotropic prior's direction edge sums keep three partials per component
  h->d_hpart = (double*)A((size_t)hyper_grid(N) * D * (o.w_prior == BFMRI_PRIOR_ANISO ? 3 : 1) * sizeof(double));
  h->d_bar = (unsigned int*)A(2 * sizeof(unsigned int));
  h->d_err = (int*)A(sizeof(int));
  h->d_ctrl = (PcgCtrl*)A(3 * sizeof(PcgCtrl));
  h->d_flags = (int*)A(4 * sizeof(int));
  h->d_edge = (double*)A((size_t)3 * D * ld * sizeof(double));
  if (o.w_prior == BFMRI_PRIOR_LTL) h->d_lt = (double*)A((size_t)K * ld * sizeof(double));
  if (o.w_prior == BFMRI_PRIOR_ANISO) {
    h->d_alpha3 = (double*)A(3 * (size_t)K * sizeof(double));
    h->d_prop3 = (double*)A(3 * (size_t)K * sizeof(double));
    h->d_waux = (double*)A((size_t)K * ld * sizeof(double));
    h->d_qdir = (double*)A(6 * (size_t)K * sizeof(double));
    h->d_loga = (double*)A((size_t)K * sizeof(double));
    h->d_alam = (double*)A((size_t)K * sizeof(double));
    h->d_acc = (long long*)A((size_t)K * sizeof(long long));
  }
  if (!h->d_edge || (o.w_prior == BFMRI_PRIOR_LTL && !h->d_lt) ||
      (o.w_prior == BFMRI_PRIOR_ANISO &&
       (!h->d_alpha3 || !h->d_prop3 || !h->d_waux || !h->d_qdir || !h->d_loga || !h->d_alam || !h->d_acc))) {
    bfmri_destroy(h);
    return fail(nullptr, BFMRI_ERR_OOM, "device allocation failed");
  }
  if (o.precision == BFMRI_PREC_MIXED) {
    h->d_blocks32 = (float*)A((size_t)ntri(D) * ld * sizeof(float));
    h->d_mfac32 = (float*)A((size_t)ntri(D) * ld * sizeof(float));
    float** f32[] = {&h->d_u32, &h->d_r32, &h->d_w32, &h->d_p32, &h->d_s32, &h->d_d32};
    for (float** pp : f32) *pp = (float*)A((size_t)D * ld * sizeof(float));
    if (!h->d_blocks32 || !h->d_mfac32 || !h->d_u32 || !h->d_r32 || !h->d_w32 || !h->d_p32 ||
        !h->d_s32 || !h->d_d32) {
      bfmri_destroy(h);
      return fail(nullptr, BFMRI_ERR_OOM, "device allocation failed");
    }
  }
  void* must[] = {h->d_nbr, h->d_lin, h->d_red, h->d_black, h->d_colour, h->d_sweep_ctr, h->d_Y, h->d_X, h->d_stats, h->d_Sxx, h->d_W, h->d_A,
                  h->d_lam, h->d_alpha, h->d_beta, h->d_G, h->d_blocks, h->d_mfac, h->d_rhs,
                  h->d_bmean, h->d_r, h->d_z, h->d_q, h->d_p0, h->d_p1, h->d_part, h->d_hpart,
                  h->d_bar, h->d_err, h->d_ctrl, h->d_flags};
  for (void* p : must) {
    if (!p) {
      bfmri_destroy(h);
      return fail(nullptr, BFMRI_ERR_OOM, "device allocation failed");
    }
  }
  cudaStream_t s = h->stream;
  cudaError_t e = cudaSuccess;
  std::vector<int> linp(ld, 0), red, black;
  std::vector<unsigned char> colour(ld, 0);
  for (int n = 0; n < N; ++n) {
    linp[n] = lin[n];
    const long long l = lin[n];
    const long long xyz = l % lat->nx + (l / lat->nx) % lat->ny + l / ((long long)lat->nx * lat->ny);
    colour[n] = (unsigned char)(xyz % 2);
    (xyz % 2 == 0 ? red : black).push_back(n);
  }
  h->n_red = (int)red.size();
  h->n_black = (int)black.size();
  h->colour_host.assign(colour.begin(), colour.begin() + N);
  if (!e) e = cudaMemcpyAsync(h->d_colour, colour.data(), ld, cudaMemcpyHostToDevice, s);
  if (!e && !red.empty()) e = cudaMemcpyAsync(h->d_red, red.data(), red.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  if (!e && !black.empty()) e = cudaMemcpyAsync(h->d_black, black.data(), black.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(h->d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(h->d_lin, linp.data(), ld * sizeof(int), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(h->d_Y, ysrc, (size_t)T * N * esz, cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(h->d_X, X, (size_t)T * K * sizeof(double), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(h->d_Sxx, h->Sxx.data(), h->Sxx.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  // prior means (Appendix C, trick 2); W = 0, A = 0
  std::vector<double> init((size_t)D * ld, 0.0);
  if (!e) e = cudaMemcpyAsync(h->d_W, init.data(), (size_t)K * ld * sizeof(double), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(h->d_A, init.data(), (size_t)Pa * ld * sizeof(double), cudaMemcpyHostToDevice, s);
  std::vector<double> lam0(ld, o.u1 * o.u2), al0(K, o.q1 * o.q2), be0(Pa, o.r1 * o.r2);
  if (!e) e = cudaMemcpyAsync(h->d_lam, lam0.data(), ld * sizeof(double), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(h->d_alpha, al0.data(), K * sizeof(double), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(h->d_beta, be0.data(), Pa * sizeof(double), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemsetAsync(h->d_ctrl, 0, 3 * sizeof(PcgCtrl), s);
  if (!e && h->d_alpha3) {
    std::vector<double> a3(3 * (size_t)K, o.q1 * o.q2);
    e = cudaMemcpyAsync(h->d_alpha3, a3.data(), a3.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemsetAsync(h->d_acc, 0, K * sizeof(long long), s);
    if (!e) e = cudaMemsetAsync(h->d_qdir, 0, 6 * (size_t)K * sizeof(double), s);
    if (!e) e = cudaMemsetAsync(h->d_loga, 0, K * sizeof(double), s);
    if (!e) e = cudaMemsetAsync(h->d_alam, 0, K * sizeof(double), s);
    if (!e) e = cudaMemsetAsync(h->d_waux, 0, (size_t)K * ld * sizeof(double), s);
  }
  if (!e) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    std::string msg = std::string("bfmri_create: ") + cudaGetErrorString(e);
    bfmri_destroy(h);
    return fail(nullptr, BFMRI_ERR_CUDA, msg);
  }
  *out = h;
  return BFMRI_OK;
}

namespace {
bfmri_status drop_sweep_graph(bfmri_handle* h);
}  // namespace

bfmri_status bfmri_set_edge_factors(bfmri_handle* h, const float* factors) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (!factors) {
    RET(drop_sweep_graph(h));
    if (h->d_ce) dfree(h, h->d_ce);
    h->d_ce = nullptr;
    return BFMRI_OK;
  }
  if ((h->opt.precond != BFMRI_PRECOND_NONE && h->opt.precond != BFMRI_PRECOND_BLOCK_JACOBI &&
       h->opt.precond != BFMRI_PRECOND_RB_REDUCED) ||
      h->opt.precision != BFMRI_PREC_FP64 || h->opt.w_prior != BFMRI_PRIOR_UGL)
    return fail(h, BFMRI_ERR_INVALID_ARG,
                "per-edge factors need the reduced red-black, block-Jacobi or no preconditioner, FP64 "
                "and the graph-Laplacian prior");
  const size_t nsite = (size_t)h->nx * h->ny * h->nz, ld = h->ld;
  std::vector<unsigned short> planes(3 * ld, (unsigned short)0x3F80);   // BF16 1.0 in the padding
  for (int d = 0; d < h->ndir / 2; ++d)   // the z plane is not read with 4 neighbours
    for (int n = 0; n < h->N; ++n) {
      const float f = factors[(size_t)d * nsite + (size_t)h->lin_host[n]];
      if (!(f > 0.0f) || !std::isfinite(f)) return fail(h, BFMRI_ERR_INVALID_ARG, "edge factors must be positive and finite");
      // round to the nearest BF16, ties to even
      uint32_t u;
      memcpy(&u, &f, 4);
      u += 0x7FFFu + ((u >> 16) & 1u);
      planes[(size_t)d * ld + n] = (unsigned short)(u >> 16);
    }
  RET(drop_sweep_graph(h));
  if (!h->d_ce) {
    h->d_ce = (unsigned short*)dalloc(h, planes.size() * sizeof(unsigned short));
    if (!h->d_ce) return fail(h, BFMRI_ERR_OOM, "edge factor allocation failed");
  }
  CU(h, cudaMemcpyAsync(h->d_ce, planes.data(), planes.size() * sizeof(unsigned short), cudaMemcpyHostToDevice, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return BFMRI_OK;
}

bfmri_status bfmri_set_alpha_dirs(bfmri_handle* h, const double* alpha) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (!h->d_alpha3) return fail(h, BFMRI_ERR_INVALID_ARG, "alpha per direction needs the anisotropic prior");
  if (!alpha || !all_positive(alpha, 3 * (size_t)h->K))
    return fail(h, BFMRI_ERR_INVALID_ARG, "alpha per direction must be positive and finite");
  std::vector<double> a3(3 * (size_t)h->K);
  for (int k = 0; k < h->K; ++k)
    for (int d = 0; d < 3; ++d) a3[(size_t)d * h->K + k] = alpha[(size_t)k * 3 + d];
  CU(h, cudaMemcpyAsync(h->d_alpha3, a3.data(), a3.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return BFMRI_OK;
}

bfmri_status bfmri_get_alpha_dirs(bfmri_handle* h, double* alpha, long long* accepted) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (!h->d_alpha3) return fail(h, BFMRI_ERR_INVALID_ARG, "alpha per direction needs the anisotropic prior");
  std::vector<double> a3(3 * (size_t)h->K);
  CU(h, cudaMemcpyAsync(a3.data(), h->d_alpha3, a3.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (accepted)
    CU(h, cudaMemcpyAsync(accepted, h->d_acc, h->K * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (alpha)
    for (int k = 0; k < h->K; ++k)
      for (int d = 0; d < 3; ++d) alpha[(size_t)k * 3 + d] = a3[(size_t)d * h->K + k];
  return BFMRI_OK;
}

bfmri_status bfmri_aniso_last_step(bfmri_handle* h, double* Q, double* Q_aux, double* log_a, double* lam,
                                   double* w_aux) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (!h->d_alpha3) return fail(h, BFMRI_ERR_INVALID_ARG, "the exchange step needs the anisotropic prior");
  const int K = h->K;
  std::vector<double> q(6 * (size_t)K);
  CU(h, cudaMemcpyAsync(q.data(), h->d_qdir, q.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (log_a) CU(h, cudaMemcpyAsync(log_a, h->d_loga, K * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (lam) CU(h, cudaMemcpyAsync(lam, h->d_alam, K * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < K; ++k)
    for (int d = 0; d < 3; ++d) {
      if (Q) Q[(size_t)k * 3 + d] = q[(size_t)d * K + k];
      if (Q_aux) Q_aux[(size_t)k * 3 + d] = q[(size_t)(3 + d) * K + k];
    }
  if (w_aux) RET(to_host(h, w_aux, h->d_waux, K));
  return BFMRI_OK;
}

bfmri_status bfmri_destroy(bfmri_handle* h) {
  if (!h) return BFMRI_OK;
  cudaStreamSynchronize(h->stream);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  if (h->sweep_exec) cudaGraphExecDestroy(h->sweep_exec);
  if (h->gsweep_exec) cudaGraphExecDestroy(h->gsweep_exec);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  if (h->sweep_graph) cudaGraphDestroy(h->sweep_graph);
  if (h->gsweep_graph) cudaGraphDestroy(h->gsweep_graph);
  std::vector<void*> all = h->allocs;
  for (void* p : all) dfree(h, p);
  delete h;
  return BFMRI_OK;
}

bfmri_status bfmri_precompute_stats(bfmri_handle* h) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (!h->d_Y) return fail(h, BFMRI_ERR_STATE, "statistics already computed (Y released)");
  int I = 0;
  const bool tc_ok = !h->y_f64 && stats_tc_supported(h->T, h->K, h->P, &I);
  if (h->opt.stats_kernel == BFMRI_STATS_TENSOR && !tc_ok)
    return fail(h, BFMRI_ERR_INVALID_ARG,
                "tensor-core statistics need FP32 Y, P <= 3, K <= 16 and a design that fits shared memory");
  cudaError_t e;
  if (tc_ok && h->opt.stats_kernel != BFMRI_STATS_FP64) {
    std::vector<uint16_t> dig;
    std::vector<int> exps;
    int Tpad = 0;
    stats_tc_digits(h->X_host.data(), h->T, h->K, h->P, I, dig, exps, Tpad);
    const size_t dig_bytes = (dig.size() * sizeof(uint16_t) + 255) & ~size_t(255);
    unsigned char* buf = (unsigned char*)dalloc(h, dig_bytes + 256 + exps.size() * sizeof(int));
    if (!buf) return fail(h, BFMRI_ERR_OOM, "device allocation failed");
    int* d_err = reinterpret_cast<int*>(buf + dig_bytes);
    int* d_exp = d_err + 64;
    e = cudaMemcpyAsync(buf, dig.data(), dig.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_exp, exps.data(), exps.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), h->stream);
    StatsTcArgs a;
    a.N = h->N;
    a.T = h->T;
    a.K = h->K;
    a.P = h->P;
    a.ld = h->ld;
    a.Y = static_cast<const float*>(h->d_Y);
    a.X = h->d_X;
    a.xdig = reinterpret_cast<const uint16_t*>(buf);
    a.xexp = d_exp;
    a.stats = h->d_stats;
    a.I = I;
    a.Tpad = Tpad;
    a.groups = (h->K + 7) / 8;
    a.sm_cap = h->opt.sm_budget;
    a.err = d_err;
    if (e == cudaSuccess) {
      Timed tm(h, BFMRI_T_STATS);
      e = launch_stats_tc(a, h->stream);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dfree(h, buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "stats (tensor cores)");
    if (herr != 0)
      return fail(h, BFMRI_ERR_TIMEOUT, "tensor-core statistics: a pipeline wait gave up (stage " +
                                            std::to_string(herr) + ")");
  } else {
    StatsArgs a;
    a.N = h->N;
    a.T = h->T;
    a.K = h->K;
    a.P = h->P;
    a.ld = h->ld;
    a.Y = h->d_Y;
    a.y_is_f64 = h->y_f64;
    a.X = h->d_X;
    a.stats = h->d_stats;
    {
      Timed tm(h, BFMRI_T_STATS);
      e = launch_stats(a, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "stats");
    CU(h, cudaStreamSynchronize(h->stream));
  }
  dfree(h, h->d_Y);
  h->d_Y = nullptr;
  h->stats_ready = true;
  return BFMRI_OK;
}

bfmri_status bfmri_get_stats(bfmri_handle* h, double* out) {
  RET(require_stats(h));
  if (!out) return fail(h, BFMRI_ERR_INVALID_ARG, "out is NULL");
  const int S = n_stats(h->K, h->P);
  std::vector<double> planes((size_t)S * h->N);
  CU(h, cudaMemcpy2DAsync(planes.data(), (size_t)h->N * sizeof(double), h->d_stats,
                          h->ld * sizeof(double), (size_t)h->N * sizeof(double), S,
                          cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  for (int n = 0; n < h->N; ++n)
    for (int j = 0; j < S; ++j) out[(size_t)n * S + j] = planes[(size_t)j * h->N + n];
  return BFMRI_OK;
}

bfmri_status bfmri_set_state(bfmri_handle* h, const double* W, const double* A,
                             const double* lambda, const double* alpha, const double* beta) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (W && !all_finite(W, (size_t)h->K * h->N)) return fail(h, BFMRI_ERR_INVALID_ARG, "W not finite");
  if (A && !all_finite(A, (size_t)h->P * h->N)) return fail(h, BFMRI_ERR_INVALID_ARG, "A not finite");
  if (lambda && !all_positive(lambda, h->N)) return fail(h, BFMRI_ERR_INVALID_ARG, "lambda must be > 0");
  if (alpha && !all_positive(alpha, h->K)) return fail(h, BFMRI_ERR_INVALID_ARG, "alpha must be > 0");
  if (beta && h->P > 0 && !all_positive(beta, h->P)) return fail(h, BFMRI_ERR_INVALID_ARG, "beta must be > 0");
  if (W) RET(to_dev(h, h->d_W, W, h->K));
  if (A) RET(to_dev(h, h->d_A, A, h->P));
  if (lambda) RET(to_dev(h, h->d_lam, lambda, 1));
  if (alpha) CU(h, cudaMemcpyAsync(h->d_alpha, alpha, h->K * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (alpha && h->d_alpha3) {
    // anisotropic prior: alpha_{d,k} = alpha_k for every direction
    std::vector<double> a3(3 * (size_t)h->K);
    for (int d = 0; d < 3; ++d)
      for (int k = 0; k < h->K; ++k) a3[(size_t)d * h->K + k] = alpha[k];
    CU(h, cudaMemcpyAsync(h->d_alpha3, a3.data(), a3.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
  }
  if (beta && h->P > 0)
    CU(h, cudaMemcpyAsync(h->d_beta, beta, h->P * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return BFMRI_OK;
}

bfmri_status bfmri_get_state(bfmri_handle* h, double* W, double* A, double* lambda,
                             double* alpha, double* beta) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (W) RET(to_host(h, W, h->d_W, h->K));
  if (A) RET(to_host(h, A, h->d_A, h->P));
  if (lambda) RET(to_host(h, lambda, h->d_lam, 1));
  if (alpha && h->d_alpha3) {
    RET(alpha_dir_mean(h, alpha));
  } else if (alpha) {
    CU(h, cudaMemcpyAsync(alpha, h->d_alpha, h->K * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  if (beta && h->P > 0)
    CU(h, cudaMemcpyAsync(beta, h->d_beta, h->P * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return BFMRI_OK;
}

bfmri_status bfmri_sample_W(bfmri_handle* h, uint64_t counter, double* W_out, bfmri_solve_info* info) {
  RET(require_stats(h));
  RET(begin_call(h));
  RET(enqueue_W(h, counter));
  PcgCtrl c[2];
  RET(end_call(h, c, nullptr));
  fill_info(info, c[0]);
  if (W_out) RET(to_host(h, W_out, h->d_W, h->K));
  return BFMRI_OK;
}

bfmri_status bfmri_sample_A(bfmri_handle* h, uint64_t counter, double* A_out, bfmri_solve_info* info) {
  RET(require_stats(h));
  if (h->P == 0) return BFMRI_OK;
  RET(begin_call(h));
  RET(enqueue_A(h, counter));
  PcgCtrl c[2];
  RET(end_call(h, c, nullptr));
  fill_info(info, c[1]);
  if (A_out) RET(to_host(h, A_out, h->d_A, h->P));
  return BFMRI_OK;
}

bfmri_status bfmri_sample_lambda(bfmri_handle* h, uint64_t counter, double* lambda_out) {
  RET(require_stats(h));
  RET(begin_call(h));
  RET(enqueue_gram(h));
  RET(enqueue_lambda(h, counter));
  RET(end_call(h, nullptr, nullptr));
  if (lambda_out) RET(to_host(h, lambda_out, h->d_lam, 1));
  return BFMRI_OK;
}

bfmri_status bfmri_sample_alpha(bfmri_handle* h, uint64_t counter, double* alpha_out) {
  RET(require_stats(h));
  RET(begin_call(h));
  RET(enqueue_hyper(h, counter, false));
  RET(end_call(h, nullptr, nullptr));
  if (alpha_out && h->d_alpha3) {
    RET(alpha_dir_mean(h, alpha_out));
  } else if (alpha_out) {
    CU(h, cudaMemcpy(alpha_out, h->d_alpha, h->K * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return BFMRI_OK;
}

bfmri_status bfmri_sample_beta(bfmri_handle* h, uint64_t counter, double* beta_out) {
  RET(require_stats(h));
  if (h->P == 0 || h->opt.ar_prior != BFMRI_AR_SPATIAL) return BFMRI_OK;
  RET(begin_call(h));
  RET(enqueue_hyper(h, counter, true));
  RET(end_call(h, nullptr, nullptr));
  if (beta_out) {
    CU(h, cudaMemcpy(beta_out, h->d_beta, h->P * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return BFMRI_OK;
}

bfmri_status bfmri_gibbs_sweep(bfmri_handle* h, int n_sweeps, uint64_t first_counter,
                               bfmri_sweep_info* info) {
  RET(require_stats(h));
  if (n_sweeps < 0) return fail(h, BFMRI_ERR_INVALID_ARG, "n_sweeps < 0");
  RET(begin_call(h));
  const bool spatial = h->opt.ar_prior == BFMRI_AR_SPATIAL;
  auto one_sweep = [&](uint64_t c) -> bfmri_status {
    RET(enqueue_W(h, c));
    RET(enqueue_A(h, c));
    RET(enqueue_lambda(h, c));
    RET(enqueue_hyper(h, c, false));
    if (h->P > 0 && spatial) RET(enqueue_hyper(h, c, true));
    if (h->sum.open) RET(enqueue_summary(h));
    return BFMRI_OK;
  };
  const bool graph = h->opt.use_graph && !h->opt.profile && h->opt.debug_skip_block < 0 &&
                     !h->graph_failed && n_sweeps > 0;
  if (graph && !h->sweep_exec) {
    // capture one sweep (its draws read the device counter) and one counter advance
    // captured on a private stream; the instantiated graph is launched on the handle's stream
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaSuccess;
    if (!h->capture_stream) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // begin_call's resets are done
    if (e == cudaSuccess) e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeRelaxed);
    bfmri_status cs = BFMRI_OK;
    if (e == cudaSuccess) {
      cudaStream_t user = h->stream;
      h->stream = h->capture_stream;
      h->capturing = true;
      cs = one_sweep(0);
      if (cs == BFMRI_OK) e = launch_advance_counter(h->d_sweep_ctr, h->stream);
      h->capturing = false;
      h->stream = user;
      const cudaError_t ee = cudaStreamEndCapture(h->capture_stream, &g);
      if (e == cudaSuccess) e = ee;
    }
    if (e == cudaSuccess && cs == BFMRI_OK && g) e = cudaGraphInstantiate(&h->sweep_exec, g, 0);
    if (e != cudaSuccess || cs != BFMRI_OK || !h->sweep_exec) {
      // capture is not available here: sweep with direct launches from now on (the reason is
      // kept as the handle's last message)
      h->err = std::string("CUDA graph capture unavailable, sweeps use direct launches: ") +
               (cs != BFMRI_OK ? h->err : std::string(cudaGetErrorString(e)));
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      h->sweep_exec = nullptr;
      h->graph_failed = true;
      RET(begin_call(h));
    } else {
      h->sweep_graph = g;
    }
  }
  const bool captured = graph && h->sweep_exec;
  if (captured) {
    cudaError_t e = launch_set_counter(h->d_sweep_ctr, (uint32_t)first_counter, h->stream);
    for (int s = 0; s < n_sweeps && e == cudaSuccess; ++s) e = cudaGraphLaunch(h->sweep_exec, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "captured sweep");
  } else {
    for (int s = 0; s < n_sweeps; ++s) RET(one_sweep(first_counter + (uint64_t)s));
  }
  if (h->sum.open) h->sum.n += n_sweeps;
  if (!info) {
    h->deferred = true;        // errors and counts are read by the next synchronising call
    return BFMRI_OK;
  }
  PcgCtrl c[2];
  int exhausted = 0;
  bfmri_status st = end_call(h, c, &exhausted);
  {
    info->sweeps = n_sweeps;
    info->pcg_iterations_W = c[0].iter_total;
    info->pcg_iterations_A = c[1].iter_total;
    info->last_rel_residual_W = c[0].rel_res;
    info->gamma_exhausted = exhausted;
    info->captured = captured ? 1 : 0;
  }
  return st;
}

bfmri_status bfmri_synchronize(bfmri_handle* h, bfmri_sweep_info* info) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  PcgCtrl c[2];
  int exhausted = 0;
  const bool was_deferred = h->deferred;
  if (!was_deferred) {
    // nothing unread: wait for the stream; the counters are those of no work
    CU(h, cudaStreamSynchronize(h->stream));
    if (info) memset(info, 0, sizeof(*info));
    return BFMRI_OK;
  }
  const bfmri_status st = end_call(h, c, &exhausted);
  if (info) {
    memset(info, 0, sizeof(*info));
    info->pcg_iterations_W = c[0].iter_total;
    info->pcg_iterations_A = c[1].iter_total;
    info->last_rel_residual_W = c[0].rel_res;
    info->gamma_exhausted = exhausted;
  }
  return st;
}

namespace {

// Table entry of one right-hand side of a grouped launch, with handle h's lattice.
MrhsRhsPtrs rhs_entry(const bfmri_handle* h, const void* blocks, const void* mfac,
                      const double* scale, const void* b, void* x) {
  MrhsRhsPtrs t{};
  t.blocks = blocks;
  t.mfac = mfac;
  t.scale = scale;
  t.b = b;
  t.x = x;
  t.N = h->N;
  t.ndir = h->ndir;
  t.ld = h->ld;
  t.nbr = h->d_nbr;
  t.red = h->d_red;
  t.black = h->d_black;
  t.n_red = h->n_red;
  t.n_black = h->n_black;
  for (int d = 0; d < 3; ++d) t.cw[d] = h->opt.edge_weight[d];
  return t;
}

bool same_lattice(const bfmri_handle* a, const bfmri_handle* b) {
  return a->nx == b->nx && a->ny == b->ny && a->nz == b->nz && a->ndir == b->ndir && a->N == b->N &&
         a->ld == b->ld && a->mask_hash == b->mask_hash;
}

// Log-det probes of one handle's W system that ride along with the W launch of a group sweep.
struct GroupProbes {
  bfmri_handle* ph;
  int n;          // probes
  int steps;      // Lanczos steps recorded per probe
  uint64_t counter;
  double* logdet;
  double* std_err;
  double* per_probe;
};

bfmri_status group_sweep(bfmri_handle* const* hs, int n, int n_sweeps, uint64_t first_counter,
                         bfmri_sweep_info* info, const GroupProbes* gp) {
  if (!hs || n < 1 || n > 64 || n_sweeps < 0) {
    set_global_error("bfmri_gibbs_sweep_group: need 1 <= n <= 64 handles and n_sweeps >= 0");
    return BFMRI_ERR_INVALID_ARG;
  }
  for (int c = 0; c < n; ++c) {
    if (!hs[c]) {
      set_global_error("bfmri_gibbs_sweep_group: NULL handle");
      return BFMRI_ERR_INVALID_ARG;
    }
    for (int d = 0; d < c; ++d)
      if (hs[d] == hs[c]) return fail(hs[0], BFMRI_ERR_INVALID_ARG, "a handle appears twice in the group");
  }
  bfmri_handle* h0 = hs[0];
  for (int c = 0; c < n; ++c)
    if (hs[c]->opt.w_prior != BFMRI_PRIOR_UGL || hs[c]->d_ce)
      return fail(h0, BFMRI_ERR_INVALID_ARG, "grouped chains need the graph-Laplacian prior with direction weights");
  if (gp && gp->ph && (gp->ph->opt.w_prior != BFMRI_PRIOR_UGL || gp->ph->d_ce))
    return fail(h0, BFMRI_ERR_INVALID_ARG, "probes need the graph-Laplacian prior with direction weights");
  bool uneven = false;
  size_t ld_max = 0;
  int N_max = 0;
  for (int c = 0; c < n; ++c) {
    RET(require_stats(hs[c]));
    const bfmri_handle* h = hs[c];
    if (!same_lattice(h, h0)) uneven = true;
    ld_max = std::max(ld_max, h->ld);
    N_max = std::max(N_max, h->N);
    if (h->K != h0->K || h->P != h0->P || h->opt.ar_prior != h0->opt.ar_prior ||
        h->opt.delta != h0->opt.delta || h->opt.max_iter != h0->opt.max_iter ||
        h->opt.precond != h0->opt.precond ||
        (h0->opt.precond == BFMRI_PRECOND_SSOR && h->opt.ssor_omega != h0->opt.ssor_omega))
      return fail(h0, BFMRI_ERR_INVALID_ARG,
                  "grouped chains must share K, P, the AR prior, delta, max_iter and the preconditioner");
    if (h->opt.precision != BFMRI_PREC_FP64)
      return fail(h0, BFMRI_ERR_INVALID_ARG, "grouped chains solve in FP64 precision only");
  }
  const int np = gp ? gp->n : 0;
  bool ph_in_group = false;
  if (gp) {
    bfmri_handle* ph = gp->ph;
    if (!ph || np < 1 || gp->steps < 1 || n_sweeps != 1)
      return fail(h0, BFMRI_ERR_INVALID_ARG, "probes ride along with exactly one sweep: need a handle, n_probes >= 1, lanczos_steps >= 1");
    RET(require_stats(ph));
    if (ph->K != h0->K || ph->opt.precision != BFMRI_PREC_FP64)
      return fail(h0, BFMRI_ERR_INVALID_ARG, "the probe handle must have the chains' K and FP64 precision");
    for (int c = 0; c < n; ++c) ph_in_group = ph_in_group || hs[c] == ph;
    if (!same_lattice(ph, h0)) uneven = true;
    ld_max = std::max(ld_max, ph->ld);
    N_max = std::max(N_max, ph->N);
  }
  const int Sw = n + np;   // right-hand sides of the W launch that carries the probes
  if (uneven && Sw > MRHS_UNEVEN_MAX_S)
    return fail(h0, BFMRI_ERR_INVALID_ARG, "at most 128 right-hand sides in one launch over different lattices");
  if (info)
    for (int c = 0; c < n; ++c) info[c] = bfmri_sweep_info{};
  if (n_sweeps == 0) return BFMRI_OK;
  const int K = h0->K, P = h0->P;
  const bool spatial_A = P > 0 && h0->opt.ar_prior == BFMRI_AR_SPATIAL;
  RET(ensure_mrhs(h0, std::max(K, P), Sw, gp ? gp->steps : 0, ld_max, N_max));
  const int tab_len = Sw + n;   // W launch (chains, then probes), A launch
  if (gp && !h0->d_ldm) {
    h0->d_ldm = (double*)dalloc(h0, sizeof(double));
    if (!h0->d_ldm) return fail(h0, BFMRI_ERR_OOM, "probe scratch allocation failed");
  }
  if (h0->g_cap < tab_len) {
    dfree(h0, h0->d_gtab);
    dfree(h0, h0->d_gtally);
    h0->g_cap = 0;
    h0->d_gtab = (MrhsRhsPtrs*)dalloc(h0, (size_t)tab_len * sizeof(MrhsRhsPtrs));
    h0->d_gtally = (MrhsTally*)dalloc(h0, (size_t)tab_len * sizeof(MrhsTally));
    if (!h0->d_gtab || !h0->d_gtally) return fail(h0, BFMRI_ERR_OOM, "group table allocation failed");
    h0->g_cap = tab_len;
  }
  // voxel blocks and their factors (block-Jacobi, and SSOR's block diagonal)
  const bool pre = h0->opt.precond != BFMRI_PRECOND_NONE;
  const size_t vs = h0->mr_vs;
  std::vector<MrhsRhsPtrs> tab((size_t)tab_len);
  for (int c = 0; c < n; ++c) {
    bfmri_handle* h = hs[c];
    tab[c] = rhs_entry(h, h->d_blocks, pre ? h->d_mfac : nullptr, h->d_alpha, h->d_rhs, h->d_W);
    tab[Sw + c] = rhs_entry(h, h->d_blocks, pre ? h->d_mfac : nullptr, h->d_beta, h->d_rhs, h->d_A);
  }
  if (gp) {
    // probe i: b_i = L v_i with v_i Rademacher (k_probe_rhs) and x_i = 0 in the workspace,
    // preconditioned by the probe handle's block-Jacobi factor, on which log det M is built
    bfmri_handle* ph = gp->ph;
    const bool ppre = ph->opt.precond != BFMRI_PRECOND_NONE;
    for (int i = 0; i < np; ++i)
      tab[n + i] = rhs_entry(ph, ph->d_blocks, ppre ? ph->d_mfac : nullptr, ph->d_alpha,
                             h0->mr_b + (size_t)(n + i) * vs, h0->mr_x + (size_t)(n + i) * vs);
  }
  cudaStream_t st0 = h0->stream;
  CU(h0, cudaMemcpyAsync(h0->d_gtab, tab.data(), tab.size() * sizeof(MrhsRhsPtrs), cudaMemcpyHostToDevice, st0));
  CU(h0, cudaMemsetAsync(h0->d_gtally, 0, (size_t)tab_len * sizeof(MrhsTally), st0));
  // every chain's work (and the probe handle's) goes to the first handle's stream for the
  // duration of the call
  std::vector<bfmri_handle*> all(hs, hs + n);
  if (gp && !ph_in_group) all.push_back(gp->ph);
  std::vector<cudaStream_t> saved(all.size());
  for (size_t c = 0; c < all.size(); ++c) {
    saved[c] = all[c]->stream;
    all[c]->stream = st0;
  }
  ProbeArgs pa{};
  if (gp) {
    bfmri_handle* ph = gp->ph;
    pa.N = ph->N;
    pa.ld = ph->ld;
    pa.ndir = ph->ndir;
    pa.f32 = 0;
    pa.nbr = ph->d_nbr;
    pa.lin = ph->d_lin;
    pa.mfac = nullptr;
    pa.mfac64 = ph->opt.precond != BFMRI_PRECOND_NONE ? ph->d_mfac : nullptr;
    pa.S = np;
    pa.vs = vs;
    pa.b = h0->mr_b + (size_t)n * vs;
    pa.x = h0->mr_x + (size_t)n * vs;
    pa.rng = rng_of(ph, gp->counter, TAG_PROBE);
    for (int d = 0; d < 3; ++d) pa.cw[d] = ph->opt.edge_weight[d];
    pa.tile = 1;
  }
  auto solve = [&](int D, int which, bool probes) -> bfmri_status {
    const int S = probes ? Sw : n;
    MrhsArgs m = mrhs_args(h0, D, S, nullptr, h0->opt.max_iter, false);
    mrhs_ssor(h0, m);
    if (probes) {
      // the probes' Lanczos quadrature needs plain block-Jacobi PCG: the whole launch uses it
      m.ssor = 0;
      m.reduced = 0;
      m.hist = h0->mr_hist;
      m.hist_len = gp->steps;
      m.max_iter = std::max(h0->opt.max_iter, gp->steps);
    }
    m.N = N_max;
    m.uneven = uneven ? 1 : 0;
    m.tab = h0->d_gtab + (which == 0 ? 0 : (size_t)Sw);
    m.tally = h0->d_gtally + (which == 0 ? 0 : (size_t)Sw);
    m.blocks = nullptr;
    m.mfac = nullptr;
    m.b = nullptr;
    m.x = nullptr;
    Timed tm(h0, which == 0 ? BFMRI_T_PCG_W : BFMRI_T_PCG_A);
    const cudaError_t e = launch_mrhs(D, m, st0, nullptr);
    if (e != cudaSuccess) return cuda_fail(h0, e, "grouped multi-RHS PCG");
    return BFMRI_OK;
  };
  bfmri_status st = BFMRI_OK;
  for (size_t c = 0; c < all.size() && st == BFMRI_OK; ++c) st = begin_call(all[c]);
  // one sweep of every chain, W launch carrying the probes when asked
  auto one_sweep = [&](uint64_t cnt, bool probes) -> bfmri_status {
    bfmri_status st = BFMRI_OK;
    for (int c = 0; c < n && st == BFMRI_OK; ++c) st = assemble_W(hs[c], cnt);
    if (probes && st == BFMRI_OK) {
      bfmri_handle* ph = gp->ph;
      if (!ph_in_group) {
        // the probe handle's W system at its current state, without perturbation
        AssembleArgs aa = assemble_args(ph, ph->d_alpha, 0, TAG_W);
        aa.perturb = 0;
        aa.blocks32 = nullptr;
        aa.mfac32 = nullptr;
        const cudaError_t e = launch_assemble_w(aa, st0);
        if (e != cudaSuccess) st = cuda_fail(h0, e, "assemble (probes)");
      }
      if (st == BFMRI_OK) {
        const cudaError_t e = launch_probe(K, pa, 0, nullptr, st0);
        if (e != cudaSuccess) st = cuda_fail(h0, e, "probe right-hand sides");
      }
    }
    if (st == BFMRI_OK) st = solve(K, 0, probes);
    if (probes && st == BFMRI_OK && pa.mfac64) {
      // log det M from the probe handle's block-Jacobi factor, before a chain's A step
      // reuses the factor's storage: per-voxel terms, summed in a fixed order
      cudaError_t e = launch_probe(K, pa, 1, h0->mr_out, st0);
      if (e == cudaSuccess) e = launch_sum_columns(h0->mr_out, gp->ph->N, 1, h0->d_ldm, st0);
      if (e != cudaSuccess) st = cuda_fail(h0, e, "logdet M");
    }
    for (int c = 0; c < n && st == BFMRI_OK; ++c) st = assemble_A(hs[c], cnt);
    if (st == BFMRI_OK && spatial_A) st = solve(P, 1, false);
    for (int c = 0; c < n && st == BFMRI_OK; ++c) {
      bfmri_handle* h = hs[c];
      st = enqueue_lambda(h, cnt);
      if (st == BFMRI_OK) st = enqueue_hyper(h, cnt, false);
      if (st == BFMRI_OK && spatial_A) st = enqueue_hyper(h, cnt, true);
      if (st == BFMRI_OK && h->sum.open) st = enqueue_summary(h);
    }
    return st;
  };
  // CUDA graph of one group sweep (options.use_graph on the first chain): captured once for
  // this list of chains and workspace, its draws reading each chain's device counter, then
  // replayed once per sweep; not with probes, per-launch timing, summaries or the test hook
  bool graph = !gp && h0->opt.use_graph && !h0->gsweep_failed;
  for (int c = 0; c < n && graph; ++c)
    graph = !hs[c]->opt.profile && hs[c]->opt.debug_skip_block < 0 && !hs[c]->sum.open;
  std::vector<uint64_t> uids((size_t)n);
  for (int c = 0; c < n; ++c) uids[c] = hs[c]->uid;
  if (graph && st == BFMRI_OK && (!h0->gsweep_exec || h0->gsweep_uids != uids || h0->gsweep_ws != h0->mr_r)) {
    if (h0->gsweep_exec) cudaGraphExecDestroy(h0->gsweep_exec);
    if (h0->gsweep_graph) cudaGraphDestroy(h0->gsweep_graph);
    h0->gsweep_exec = nullptr;
    h0->gsweep_graph = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaSuccess;
    if (!h0->capture_stream) e = cudaStreamCreateWithFlags(&h0->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st0);   // begin_call's resets and the table are done
    if (e == cudaSuccess) e = cudaStreamBeginCapture(h0->capture_stream, cudaStreamCaptureModeRelaxed);
    bfmri_status cs = BFMRI_OK;
    if (e == cudaSuccess) {
      const cudaStream_t saved0 = st0;
      st0 = h0->capture_stream;
      for (int c = 0; c < n; ++c) {
        hs[c]->stream = st0;
        hs[c]->capturing = true;
      }
      cs = one_sweep(0, false);
      for (int c = 0; c < n && cs == BFMRI_OK && e == cudaSuccess; ++c)
        e = launch_advance_counter(hs[c]->d_sweep_ctr, st0);
      for (int c = 0; c < n; ++c) {
        hs[c]->capturing = false;
        hs[c]->stream = saved0;
      }
      st0 = saved0;
      const cudaError_t ee = cudaStreamEndCapture(h0->capture_stream, &g);
      if (e == cudaSuccess) e = ee;
    }
    if (e == cudaSuccess && cs == BFMRI_OK && g) e = cudaGraphInstantiate(&h0->gsweep_exec, g, 0);
    if (e != cudaSuccess || cs != BFMRI_OK || !h0->gsweep_exec) {
      h0->err = std::string("CUDA graph capture unavailable, group sweeps use direct launches: ") +
                (cs != BFMRI_OK ? h0->err : std::string(cudaGetErrorString(e)));
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      h0->gsweep_exec = nullptr;
      h0->gsweep_failed = true;
      graph = false;
    } else {
      h0->gsweep_graph = g;
      h0->gsweep_uids = uids;
      h0->gsweep_ws = h0->mr_r;
    }
  }
  if (graph && st == BFMRI_OK && h0->gsweep_exec) {
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < n && e == cudaSuccess; ++c)
      e = launch_set_counter(hs[c]->d_sweep_ctr, (uint32_t)first_counter, st0);
    for (int sw = 0; sw < n_sweeps && e == cudaSuccess; ++sw) e = cudaGraphLaunch(h0->gsweep_exec, st0);
    if (e != cudaSuccess) st = cuda_fail(h0, e, "captured group sweep");
  } else {
    for (int sw = 0; sw < n_sweeps && st == BFMRI_OK; ++sw)
      st = one_sweep(first_counter + (uint64_t)sw, gp != nullptr && sw == 0);
  }
  for (int c = 0; c < n; ++c)
    if (hs[c]->sum.open) hs[c]->sum.n += n_sweeps;
  std::vector<int> exhausted(all.size(), 0);
  for (size_t c = 0; c < all.size(); ++c) {
    const bfmri_status sc = end_call(all[c], nullptr, &exhausted[c]);
    if (st == BFMRI_OK) st = sc;
  }
  for (size_t c = 0; c < all.size(); ++c) all[c]->stream = saved[c];
  if (st != BFMRI_OK) return st;
  std::vector<MrhsTally> tally((size_t)tab_len);
  CU(h0, cudaMemcpy(tally.data(), h0->d_gtally, tally.size() * sizeof(MrhsTally), cudaMemcpyDeviceToHost));
  for (int c = 0; c < n; ++c) {
    if (info) {
      info[c].sweeps = n_sweeps;
      info[c].pcg_iterations_W = tally[c].iters;
      info[c].pcg_iterations_A = spatial_A ? tally[Sw + c].iters : 0;
      info[c].last_rel_residual_W = tally[c].rel_res;
      info[c].gamma_exhausted = exhausted[c];
    }
    for (int w = 0; w < (spatial_A ? 2 : 1); ++w) {
      const int code = tally[(size_t)(w ? Sw : 0) + c].status_any;
      const std::string who = "chain " + std::to_string(c) + (w ? " (A)" : " (W)");
      if (code == 4) return fail(h0, BFMRI_ERR_NOT_CONVERGED, "PCG reached max_iter in " + who);
      if (code == 3) return fail(h0, BFMRI_ERR_NOT_SPD, "PCG breakdown (p'Bp <= 0) in " + who);
      if (code == 7) return fail(h0, BFMRI_ERR_INVALID_ARG, "non-finite value in PCG of " + who);
    }
  }
  if (!gp) return BFMRI_OK;
  // the probes: states and CG coefficients of right-hand sides n .. n + np - 1
  bfmri_handle* ph = gp->ph;
  std::vector<RhsState> pst((size_t)np);
  CU(h0, cudaMemcpy(pst.data(), h0->mr_st + n, (size_t)np * sizeof(RhsState), cudaMemcpyDeviceToHost));
  for (int i = 0; i < np; ++i) {
    if (pst[i].status == 3) return fail(h0, BFMRI_ERR_NOT_SPD, "probe solve breakdown");
    if (pst[i].status == 7) return fail(h0, BFMRI_ERR_INVALID_ARG, "non-finite value in probe solve");
    if (pst[i].status == 4) return fail(h0, BFMRI_ERR_NOT_CONVERGED, "probe solve reached max_iter");
  }
  std::vector<double> hist((size_t)gp->steps * Sw * 2);
  CU(h0, cudaMemcpy(hist.data(), h0->mr_hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost));
  double ldm = 0.0;
  if (pa.mfac64) CU(h0, cudaMemcpy(&ldm, h0->d_ldm, sizeof(double), cudaMemcpyDeviceToHost));
  const double vnorm2 = (double)K * ph->N;
  std::vector<double> est((size_t)np, 0.0);
  for (int i = 0; i < np; ++i) {
    const int mi = std::min(pst[i].iters, gp->steps);
    if (mi < 1) continue;
    std::vector<double> al(mi), be(mi);
    for (int j = 0; j < mi; ++j) {
      al[j] = hist[((size_t)j * Sw + n + i) * 2 + 0];
      be[j] = hist[((size_t)j * Sw + n + i) * 2 + 1];
    }
    double q = 0.0;
    const bfmri_status qs = bfmri_lanczos_log_quadrature(mi, al.data(), be.data(), &q);
    if (qs != BFMRI_OK) return fail(h0, qs, "Lanczos quadrature failed");
    est[i] = vnorm2 * q;
  }
  double mean = 0.0;
  for (double v : est) mean += v;
  mean /= np;
  double var = 0.0;
  for (double v : est) var += (v - mean) * (v - mean);
  if (gp->logdet) *gp->logdet = ldm + mean;
  if (gp->std_err) *gp->std_err = np > 1 ? std::sqrt(var / (np - 1) / np) : 0.0;
  if (gp->per_probe)
    for (int i = 0; i < np; ++i) gp->per_probe[i] = est[i];
  return BFMRI_OK;
}

}  // namespace

bfmri_status bfmri_gibbs_sweep_group(bfmri_handle* const* hs, int n, int n_sweeps,
                                     uint64_t first_counter, bfmri_sweep_info* info) {
  return group_sweep(hs, n, n_sweeps, first_counter, info, nullptr);
}

bfmri_status bfmri_gibbs_sweep_group_probes(bfmri_handle* const* hs, int n, uint64_t counter,
                                            bfmri_handle* probe_handle, int n_probes,
                                            int lanczos_steps, uint64_t probe_counter,
                                            double* logdet, double* std_err, double* per_probe,
                                            bfmri_sweep_info* info) {
  if (n_probes < 1 || n_probes > 127) {
    set_global_error("bfmri_gibbs_sweep_group_probes: need 1 <= n_probes <= 127");
    return BFMRI_ERR_INVALID_ARG;
  }
  GroupProbes gp{probe_handle, n_probes, lanczos_steps, probe_counter, logdet, std_err, per_probe};
  return group_sweep(hs, n, 1, counter, info, &gp);
}

namespace {

// A captured sweep holds the launches it was captured with: opening or closing a summary
// changes them, so the next sweep captures again.
bfmri_status drop_sweep_graph(bfmri_handle* h) {
  if (!h->sweep_exec && !h->sweep_graph) return BFMRI_OK;
  CU(h, cudaStreamSynchronize(h->stream));
  if (h->sweep_exec) cudaGraphExecDestroy(h->sweep_exec);
  if (h->sweep_graph) cudaGraphDestroy(h->sweep_graph);
  h->sweep_exec = nullptr;
  h->sweep_graph = nullptr;
  return BFMRI_OK;
}

void free_summary(bfmri_handle* h) {
  auto& m = h->sum;
  for (void* p : {(void*)m.ref, (void*)m.S1, (void*)m.S2, (void*)m.C, (void*)m.gamma, (void*)m.mean,
                  (void*)m.cov, (void*)m.ppm, (void*)m.count, (void*)m.in_set, (void*)m.joint,
                  (void*)m.scratch})
    dfree(h, p);
  m = bfmri_handle::Summary{};
}

bool contrasts_ok(int nc, int K, const double* C, const double* gamma) {
  if (nc < 0 || nc > MAX_CONTRASTS) return false;
  if (nc == 0) return true;
  if (!C || !gamma) return false;
  for (int i = 0; i < nc * K; ++i)
    if (!std::isfinite(C[i])) return false;
  for (int i = 0; i < nc; ++i)
    if (std::isnan(gamma[i])) return false;
  return true;
}

}  // namespace

bfmri_status bfmri_summary_begin(bfmri_handle* h, int n_contrasts, const double* C,
                                 const double* gamma, const int* joint_set, int n_joint) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  const int K = h->K, nc = n_contrasts;
  if (!contrasts_ok(nc, K, C, gamma))
    return fail(h, BFMRI_ERR_INVALID_ARG, "contrasts: 0 <= n_contrasts <= 16, finite C, gamma not NaN");
  if (n_joint < 0 || (n_joint > 0 && !joint_set))
    return fail(h, BFMRI_ERR_INVALID_ARG, "joint set: n_joint < 0 or joint_set missing");
  for (int i = 0; i < n_joint; ++i)
    if (joint_set[i] < 0 || joint_set[i] >= h->N)
      return fail(h, BFMRI_ERR_INVALID_ARG, "joint set: voxel index out of range");
  RET(drop_sweep_graph(h));
  CU(h, cudaStreamSynchronize(h->stream));
  free_summary(h);
  const size_t ld = h->ld;
  auto& m = h->sum;
  const int ncs = std::max(nc, 1);
  m.ref = (double*)dalloc(h, (size_t)K * ld * sizeof(double));
  m.S1 = (double*)dalloc(h, (size_t)K * ld * sizeof(double));
  m.S2 = (double*)dalloc(h, (size_t)ntri(K) * ld * sizeof(double));
  m.mean = (double*)dalloc(h, (size_t)K * ld * sizeof(double));
  m.cov = (double*)dalloc(h, (size_t)ntri(K) * ld * sizeof(double));
  m.ppm = (double*)dalloc(h, (size_t)ncs * ld * sizeof(double));
  m.count = (int*)dalloc(h, (size_t)ncs * ld * sizeof(int));
  m.C = (double*)dalloc(h, (size_t)ncs * K * sizeof(double));
  m.gamma = (double*)dalloc(h, (size_t)ncs * sizeof(double));
  m.in_set = (uint8_t*)dalloc(h, ld);
  m.joint = (unsigned long long*)dalloc(h, (size_t)ncs * sizeof(unsigned long long));
  m.scratch = (unsigned int*)dalloc(h, 2 * sizeof(unsigned int));
  if (!m.ref || !m.S1 || !m.S2 || !m.mean || !m.cov || !m.ppm || !m.count || !m.C || !m.gamma ||
      !m.in_set || !m.joint || !m.scratch) {
    free_summary(h);
    return fail(h, BFMRI_ERR_OOM, "summary allocation failed");
  }
  cudaStream_t st = h->stream;
  CU(h, cudaMemcpyAsync(m.ref, h->d_W, (size_t)K * ld * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CU(h, cudaMemsetAsync(m.S1, 0, (size_t)K * ld * sizeof(double), st));
  CU(h, cudaMemsetAsync(m.S2, 0, (size_t)ntri(K) * ld * sizeof(double), st));
  CU(h, cudaMemsetAsync(m.count, 0, (size_t)ncs * ld * sizeof(int), st));
  CU(h, cudaMemsetAsync(m.joint, 0, (size_t)ncs * sizeof(unsigned long long), st));
  CU(h, cudaMemsetAsync(m.scratch, 0, 2 * sizeof(unsigned int), st));
  std::vector<uint8_t> flags(ld, 0);
  for (int i = 0; i < n_joint; ++i) flags[(size_t)joint_set[i]] = 1;
  CU(h, cudaMemcpyAsync(m.in_set, flags.data(), ld, cudaMemcpyHostToDevice, st));
  if (nc > 0) {
    CU(h, cudaMemcpyAsync(m.C, C, (size_t)nc * K * sizeof(double), cudaMemcpyHostToDevice, st));
    CU(h, cudaMemcpyAsync(m.gamma, gamma, (size_t)nc * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  CU(h, cudaStreamSynchronize(st));
  m.nc = nc;
  m.has_set = n_joint > 0;
  m.n = 0;
  m.open = true;
  return BFMRI_OK;
}

bfmri_status bfmri_summary_add(bfmri_handle* h) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (!h->sum.open) return fail(h, BFMRI_ERR_STATE, "no summary is open (bfmri_summary_begin)");
  RET(enqueue_summary(h));
  h->sum.n += 1;
  return BFMRI_OK;
}

bfmri_status bfmri_summary_get(bfmri_handle* h, long long* n_samples, double* mean, double* cov,
                               double* ppm, long long* joint_count) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  auto& m = h->sum;
  if (!m.open) return fail(h, BFMRI_ERR_STATE, "no summary is open (bfmri_summary_begin)");
  RET(end_call(h, nullptr, nullptr));   // waits; reports errors of asynchronous sweeps
  if (n_samples) *n_samples = m.n;
  if (m.n <= 0) {
    if (mean || cov || ppm || joint_count)
      return fail(h, BFMRI_ERR_STATE, "the summary holds no sample yet");
    return BFMRI_OK;
  }
  ChainFinalArgs a;
  a.g = geom(h);
  a.K = h->K;
  a.nc = m.nc;
  a.n = m.n;
  a.ref = m.ref;
  a.S1 = m.S1;
  a.S2 = m.S2;
  a.count = m.count;
  a.mean = m.mean;
  a.cov = m.cov;
  a.ppm = m.ppm;
  {
    Timed tm(h, BFMRI_T_SUMMARY);
    const cudaError_t e = launch_chain_finalize(a, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "chain summary finalize");
  }
  if (mean) RET(to_host(h, mean, m.mean, h->K));
  if (cov) RET(to_host(h, cov, m.cov, ntri(h->K)));
  if (ppm) RET(to_host(h, ppm, m.ppm, m.nc));
  if (joint_count && m.nc > 0) {
    std::vector<unsigned long long> j((size_t)m.nc);
    CU(h, cudaMemcpyAsync(j.data(), m.joint, j.size() * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    for (int c = 0; c < m.nc; ++c) joint_count[c] = (long long)j[(size_t)c];
  }
  CU(h, cudaStreamSynchronize(h->stream));
  return BFMRI_OK;
}

bfmri_status bfmri_summary_end(bfmri_handle* h) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (!h->sum.open) return BFMRI_OK;
  RET(drop_sweep_graph(h));
  CU(h, cudaStreamSynchronize(h->stream));
  free_summary(h);
  return BFMRI_OK;
}

bfmri_status bfmri_svb_summary(bfmri_handle* h, int n_contrasts, const double* C,
                               const double* gamma, double* mean, double* cov, double* ppm) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (h->svb_S <= 0) return fail(h, BFMRI_ERR_STATE, "no SVB samples (bfmri_spvb_step)");
  if (!contrasts_ok(n_contrasts, h->K, C, gamma))
    return fail(h, BFMRI_ERR_INVALID_ARG, "contrasts: 0 <= n_contrasts <= 16, finite C, gamma not NaN");
  const size_t ld = h->ld;
  const int K = h->K, nc = n_contrasts, ncs = std::max(nc, 1);
  // work planes: mean, packed covariance, PPMs, then the contrasts (freed on return)
  const size_t doubles = ((size_t)K + ntri(K) + ncs) * ld + (size_t)ncs * (K + 1);
  double* work = (double*)dalloc(h, doubles * sizeof(double));
  if (!work) return fail(h, BFMRI_ERR_OOM, "SVB summary allocation failed");
  double* d_mean = work;
  double* d_cov = d_mean + (size_t)K * ld;
  double* d_ppm = d_cov + (size_t)ntri(K) * ld;
  double* d_C = d_ppm + (size_t)ncs * ld;
  double* d_g = d_C + (size_t)ncs * K;
  bfmri_status st = BFMRI_OK;
  auto body = [&]() -> bfmri_status {
    RET(begin_call(h));
    if (nc > 0) {
      CU(h, cudaMemcpyAsync(d_C, C, (size_t)nc * K * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      CU(h, cudaMemcpyAsync(d_g, gamma, (size_t)nc * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    SvbSumArgs a;
    a.g = geom(h);
    a.K = K;
    a.S = h->svb_S;
    a.nc = nc;
    a.Ws = h->svb_W;
    a.C = d_C;
    a.gamma = d_g;
    a.mean = d_mean;
    a.cov = d_cov;
    a.ppm = d_ppm;
    {
      Timed tm(h, BFMRI_T_SUMMARY);
      const cudaError_t e = launch_svb_summary(a, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "SVB summary");
    }
    RET(end_call(h, nullptr, nullptr));
    if (mean) RET(to_host(h, mean, d_mean, K));
    if (cov) RET(to_host(h, cov, d_cov, ntri(K)));
    if (ppm) RET(to_host(h, ppm, d_ppm, nc));
    return BFMRI_OK;
  };
  st = body();
  cudaStreamSynchronize(h->stream);
  dfree(h, work);
  return st;
}

bfmri_status bfmri_log_joint(bfmri_handle* h, double* terms) {
  RET(require_stats(h));
  if (!terms) return fail(h, BFMRI_ERR_INVALID_ARG, "terms is NULL");
  // per-edge factors enter through the edge sums, the L'L prior through |L w_k|^2; neither's
  // pseudo-determinant depends on the sampled parameters beyond alpha's power, so the N/2
  // log alpha normaliser stands. The anisotropic prior's does (log pdet sum_d alpha_d L_d).
  if (h->opt.w_prior == BFMRI_PRIOR_ANISO)
    return fail(h, BFMRI_ERR_INVALID_ARG, "the log joint needs the graph-Laplacian or the L'L prior");
  const int K = h->K, P = h->P;
  const int grid = log_joint_grid(h->N);
  if (!h->d_lj) {
    h->d_lj = (double*)dalloc(h, (7 + (size_t)K + (size_t)P + 2 * (size_t)grid) * sizeof(double));
    if (!h->d_lj) return fail(h, BFMRI_ERR_OOM, "log joint allocation failed");
  }
  double* d_terms = h->d_lj;
  double* d_Qw = d_terms + 7;
  double* d_Qa = d_Qw + K;
  double* d_part = d_Qa + P;
  const bool spatial = P > 0 && h->opt.ar_prior == BFMRI_AR_SPATIAL;
  RET(begin_call(h));
  {
    Timed tm(h, BFMRI_T_SUMMARY);
    // quadratic forms W_k D_w W_k' and A_p D_a A_p' (the Gamma draws are skipped: out = null)
    HyperArgs q;
    q.g = geom(h);
    q.part = h->d_hpart;
    q.prior1 = q.prior2 = 0.0;
    q.out = nullptr;
    q.rng = rng_of(h, 0, TAG_ALPHA);
    q.exhausted = h->d_flags + 1;
    q.ltl = h->opt.w_prior == BFMRI_PRIOR_LTL ? 1 : 0;
    q.D = K;
    q.V = h->d_W;
    q.Q_out = d_Qw;
    cudaError_t e = launch_hyper(q, h->stream);
    if (e == cudaSuccess && spatial) {
      q.ltl = 0;   // the A prior stays the graph Laplacian
      q.D = P;
      q.V = h->d_A;
      q.Q_out = d_Qa;
      e = launch_hyper(q, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "log joint quadratic forms");
    LogJointArgs a;
    a.g = geom(h);
    a.K = K;
    a.P = P;
    a.T = h->T;
    a.spatial = spatial ? 1 : 0;
    a.stats = h->d_stats;
    a.Sxx = h->d_Sxx;
    a.W = h->d_W;
    a.A = h->d_A;
    a.lam = h->d_lam;
    a.alpha = h->d_alpha;
    a.beta = h->d_beta;
    a.Qw = d_Qw;
    a.Qa = d_Qa;
    a.u1 = h->opt.u1;
    a.u2 = h->opt.u2;
    a.q1 = h->opt.q1;
    a.q2 = h->opt.q2;
    a.r1 = h->opt.r1;
    a.r2 = h->opt.r2;
    a.part = d_part;
    a.terms = d_terms;
    e = launch_log_joint(a, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "log joint");
  }
  RET(end_call(h, nullptr, nullptr));
  CU(h, cudaMemcpyAsync(terms, d_terms, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return BFMRI_OK;
}

bfmri_status bfmri_get_timing(bfmri_handle* h, bfmri_timing* t) {
  if (!h || !t) return BFMRI_ERR_INVALID_ARG;
  RET(resolve_timing(h));
  *t = h->timing;
  return BFMRI_OK;
}

bfmri_status bfmri_reset_timing(bfmri_handle* h) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  RET(resolve_timing(h));
  memset(&h->timing, 0, sizeof(h->timing));
  return BFMRI_OK;
}

namespace {

// Autotuner of the FP32 probe solves: the right-hand-side tile (1, 2 or 4 interleaved
// right-hand sides per thread) is chosen per shape (D, S, N, SM budget) by timing each
// candidate's solve once, on the first probe call of that shape, and kept for the process.
struct TileChoice {
  int tile;
  double ms[3];
};
std::mutex g_tile_mu;
std::map<std::tuple<int, int, int, int>, TileChoice> g_tile_cache;

}  // namespace

bfmri_status bfmri_logdet_probe(bfmri_handle* h, int which, int n_probes, int lanczos_steps,
                                uint64_t counter, double* logdet, double* std_err,
                                double* traces, double* per_probe, int* iterations) {
  RET(require_stats(h));
  if ((which != 0 && which != 1) || n_probes < 1 || n_probes > 4096 || lanczos_steps < 1)
    return fail(h, BFMRI_ERR_INVALID_ARG, "bad arguments");
  const int D = which == 0 ? h->K : h->P;
  if (D == 0) return fail(h, BFMRI_ERR_INVALID_ARG, "no AR part (P = 0)");
  if ((which == 0 && h->opt.w_prior != BFMRI_PRIOR_UGL) || h->d_ce)
    return fail(h, BFMRI_ERR_INVALID_ARG, "probes need the graph-Laplacian prior with direction weights");
  RET(begin_call(h));
  const double* scale = which == 0 ? h->d_alpha : h->d_beta;
  if (which == 1 && h->opt.ar_prior != BFMRI_AR_SPATIAL) {
    static const double zeros[PMAX] = {0, 0, 0, 0};
    CU(h, cudaMemcpyAsync(h->d_bmean, zeros, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    scale = h->d_bmean;
  }
  const bool f32 = h->opt.precision == BFMRI_PREC_MIXED;
  AssembleArgs a = assemble_args(h, scale, 0, which == 0 ? TAG_W : TAG_A);
  a.perturb = 0;
  if (!f32) {
    a.blocks32 = nullptr;
    a.mfac32 = nullptr;
  }
  {
    Timed tm(h, which == 0 ? BFMRI_T_ASSEMBLE_W : BFMRI_T_ASSEMBLE_A);
    cudaError_t e = which == 0 ? launch_assemble_w(a, h->stream) : launch_assemble_a(a, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "assemble");
  }
  RET(ensure_mrhs(h, D, n_probes, lanczos_steps));
  const bool pre = h->opt.precond != BFMRI_PRECOND_NONE;
  ProbeArgs pa;
  pa.N = h->N;
  pa.ld = h->ld;
  pa.ndir = h->ndir;
  pa.f32 = f32 ? 1 : 0;
  pa.nbr = h->d_nbr;
  pa.lin = h->d_lin;
  pa.mfac = nullptr;
  pa.mfac64 = pre ? h->d_mfac : nullptr;
  pa.S = n_probes;
  pa.vs = h->mr_vs;
  pa.b = h->mr_b;
  pa.x = h->mr_x;
  pa.rng = rng_of(h, counter, TAG_PROBE);
  for (int d = 0; d < 3; ++d) pa.cw[d] = h->opt.edge_weight[d];
  pa.tile = 1;
  MrhsArgs m = mrhs_args(h, D, n_probes, scale, lanczos_steps, true);
  if (f32) {
    m.f32 = 1;
    m.blocks = h->d_blocks32;
    m.mfac = pre ? h->d_mfac32 : nullptr;
  }
  // right-hand-side tile: fixed by options.mrhs_tile, or chosen by the autotuner (FP32)
  int tile = 1;
  double tile_ms[3] = {-1.0, -1.0, -1.0};
  if (f32 && h->opt.mrhs_tile != 1) {
    if (h->opt.mrhs_tile == 2 || h->opt.mrhs_tile == 4) {
      tile = n_probes % h->opt.mrhs_tile == 0 ? h->opt.mrhs_tile : 1;
    } else {
      const auto key = std::make_tuple(D, n_probes, h->N, h->opt.sm_budget);
      bool have = false;
      {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        auto it = g_tile_cache.find(key);
        if (it != g_tile_cache.end()) {
          tile = it->second.tile;
          for (int c = 0; c < 3; ++c) tile_ms[c] = it->second.ms[c];
          have = true;
        }
      }
      if (!have) {
        const int cand[3] = {1, 2, 4};
        double best = 0.0;
        cudaEvent_t e0 = take_event(h), e1 = take_event(h);
        for (int c = 0; c < 3; ++c) {
          if (n_probes % cand[c] != 0) continue;
          pa.tile = m.tile = cand[c];
          CU(h, launch_probe(D, pa, 0, nullptr, h->stream));
          CU(h, cudaEventRecord(e0, h->stream));
          int units = 0;
          CU(h, launch_mrhs(D, m, h->stream, &units));
          CU(h, cudaEventRecord(e1, h->stream));
          CU(h, cudaEventSynchronize(e1));
          float ms = 0.f;
          CU(h, cudaEventElapsedTime(&ms, e0, e1));
          tile_ms[c] = ms;
          if (tile_ms[c] >= 0.0 && (best == 0.0 || ms < best)) {
            best = ms;
            tile = cand[c];
          }
        }
        h->event_pool.push_back(e0);
        h->event_pool.push_back(e1);
        RET(end_call(h, nullptr, nullptr));   // errors of the trial solves surface here
        RET(begin_call(h));
        std::lock_guard<std::mutex> lk(g_tile_mu);
        TileChoice tc;
        tc.tile = tile;
        for (int c = 0; c < 3; ++c) tc.ms[c] = tile_ms[c];
        g_tile_cache[key] = tc;
      }
    }
  }
  h->probe_tile = tile;
  for (int c = 0; c < 3; ++c) h->probe_tile_ms[c] = tile_ms[c];
  pa.tile = m.tile = tile;
  cudaError_t e = launch_probe(D, pa, 0, nullptr, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "probe rhs");
  {
    Timed tm(h, BFMRI_T_OTHER, true, 0);
    int units = 0;
    e = launch_mrhs(D, m, h->stream, &units);
    if (e != cudaSuccess) return cuda_fail(h, e, "multi-RHS PCG");
  }
  RET(end_call(h, nullptr, nullptr));
  std::vector<RhsState> st(n_probes);
  CU(h, cudaMemcpy(st.data(), h->mr_st, n_probes * sizeof(RhsState), cudaMemcpyDeviceToHost));
  if (iterations)
    for (int i = 0; i < n_probes; ++i) iterations[i] = st[i].total;
  for (int i = 0; i < n_probes; ++i) {
    if (st[i].status == 4) return fail(h, BFMRI_ERR_NOT_CONVERGED, "probe solve reached lanczos_steps");
    if (st[i].status == 3) return fail(h, BFMRI_ERR_NOT_SPD, "probe solve breakdown");
    if (st[i].status != 0) return fail(h, BFMRI_ERR_INVALID_ARG, "non-finite value in probe solve");
  }
  std::vector<double> hist((size_t)lanczos_steps * n_probes * 2);
  CU(h, cudaMemcpy(hist.data(), h->mr_hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost));
  // log det M
  double ldm = 0.0;
  if (pre) {
    // per-voxel terms, summed on the device into h->d_hpart[0]
    e = launch_probe(D, pa, 1, h->mr_out, h->stream);
    if (e == cudaSuccess) e = launch_sum_columns(h->mr_out, h->N, 1, h->d_hpart, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "logdet M");
    CU(h, cudaMemcpyAsync(&ldm, h->d_hpart, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
  }
  // Lanczos quadrature per probe
  const double vnorm2 = (double)D * h->N;
  std::vector<double> est(n_probes);
  for (int i = 0; i < n_probes; ++i) {
    const int mi = std::min(st[i].iters, lanczos_steps);
    if (mi < 1) {
      est[i] = 0.0;
      continue;
    }
    std::vector<double> al(mi), be(mi);
    for (int j = 0; j < mi; ++j) {
      al[j] = hist[((size_t)j * n_probes + i) * 2 + 0];
      be[j] = hist[((size_t)j * n_probes + i) * 2 + 1];
    }
    double q = 0.0;
    bfmri_status qs = bfmri_lanczos_log_quadrature(mi, al.data(), be.data(), &q);
    if (qs != BFMRI_OK) return fail(h, qs, "Lanczos quadrature failed");
    est[i] = vnorm2 * q;
  }
  double mean = 0.0;
  for (double v : est) mean += v;
  mean /= n_probes;
  double var = 0.0;
  for (double v : est) var += (v - mean) * (v - mean);
  if (logdet) *logdet = ldm + mean;
  if (std_err) *std_err = n_probes > 1 ? std::sqrt(var / (n_probes - 1) / n_probes) : 0.0;
  if (per_probe)
    for (int i = 0; i < n_probes; ++i) per_probe[i] = est[i];
  if (traces) {
    // partials [gx][n_probes][D], summed over gx on the device (the column sums go to the
    // part of mr_out after the partials), then over the probes on the host
    e = launch_probe(D, pa, 2, h->mr_out, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "traces");
    const int gx = (h->N + 127) / 128;
    const size_t C = (size_t)n_probes * D;
    double* colsum = h->mr_out + (size_t)gx * C;
    e = launch_sum_columns(h->mr_out, gx, (int)C, colsum, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "traces");
    std::vector<double> part(C);
    CU(h, cudaMemcpyAsync(part.data(), colsum, C * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < D; ++k) {
      double t = 0.0;
      for (int i = 0; i < n_probes; ++i) t += part[(size_t)i * D + k];
      traces[k] = t / n_probes;
    }
  }
  return BFMRI_OK;
}

bfmri_status bfmri_spvb_step(bfmri_handle* h, int n_samples, uint64_t counter, int extrapolate,
                             double* alpha_vb, double* beta_vb, bfmri_svb_info* info) {
  RET(require_stats(h));
  if (n_samples < 1 || n_samples > 4096) return fail(h, BFMRI_ERR_INVALID_ARG, "n_samples must be in [1, 4096]");
  if (h->opt.w_prior != BFMRI_PRIOR_UGL || h->d_ce)
    return fail(h, BFMRI_ERR_INVALID_ARG, "the SVB step needs the graph-Laplacian prior with direction weights");
  const int K = h->K, P = h->P, S = n_samples;
  const size_t ld = h->ld;
  const bool spatial = h->opt.ar_prior == BFMRI_AR_SPATIAL;
  // (re)size the sample store; new samples start from the current W and A
  if (S != h->svb_S) {
    double* nW = (double*)dalloc(h, (size_t)S * K * ld * sizeof(double));
    double* nA = (double*)dalloc(h, (size_t)S * std::max(P, 1) * ld * sizeof(double));
    if (!nW || !nA) return fail(h, BFMRI_ERR_OOM, "SVB sample allocation failed");
    for (int j = 0; j < S; ++j) {
      const bool keep = j < h->svb_S;
      CU(h, cudaMemcpyAsync(nW + (size_t)j * K * ld, keep ? h->svb_W + (size_t)j * K * ld : h->d_W,
                            (size_t)K * ld * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      if (P > 0)
        CU(h, cudaMemcpyAsync(nA + (size_t)j * P * ld, keep ? h->svb_A + (size_t)j * P * ld : h->d_A,
                              (size_t)P * ld * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    CU(h, cudaStreamSynchronize(h->stream));
    dfree(h, h->svb_W);
    dfree(h, h->svb_A);
    h->svb_W = nW;
    h->svb_A = nA;
    h->svb_S = S;
  }
  if (!h->svb_cmom) {
    h->svb_cmom = (double*)dalloc(h, (size_t)n_syy(P) * ld * sizeof(double));
    h->svb_gin = (double*)dalloc(h, (size_t)n_syy(P) * ld * sizeof(double));
    h->svb_ldata = (double*)dalloc(h, (size_t)ntri(h->D) * ld * sizeof(double));
    h->svb_part = (double*)dalloc(h, (size_t)1024 * h->D * sizeof(double));
    h->d_zero = (double*)dalloc(h, (size_t)(PMAX + KMAX) * sizeof(double));
    if (!h->svb_cmom || !h->svb_gin || !h->svb_ldata || !h->svb_part || !h->d_zero)
      return fail(h, BFMRI_ERR_OOM, "SVB workspace allocation failed");
    CU(h, cudaMemsetAsync(h->d_zero, 0, (PMAX + KMAX) * sizeof(double), h->stream));
  }
  RET(ensure_mrhs(h, h->D, S, 0));
  RET(begin_call(h));
  SvbArgs sv;
  memset(&sv, 0, sizeof(sv));
  sv.g = geom(h);
  sv.K = K;
  sv.P = P;
  sv.T = h->T;
  sv.S = S;
  sv.stats = h->d_stats;
  sv.Sxx = h->d_Sxx;
  sv.Ws = h->svb_W;
  sv.As = h->svb_A;
  sv.Cmom = h->svb_cmom;
  sv.Gin = h->svb_gin;
  sv.bmean = h->d_bmean;
  sv.ldata = h->svb_ldata;
  sv.u1 = h->opt.u1;
  sv.u2 = h->opt.u2;
  sv.lam = h->d_lam;
  sv.part = h->svb_part;
  sv.rhs = h->mr_b;
  cudaError_t e;
  // ---- q(W): averaged system (Eq. NFVBbB), N_s draws with fixed random numbers ----
  if (P > 0) {
    e = launch_svb(0, K, sv, h->stream, nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "svb moments");
  }
  AssembleArgs a = assemble_args(h, h->d_alpha, 0, TAG_W);
  a.perturb = 0;
  a.blocks32 = nullptr;
  a.mfac32 = nullptr;
  a.bmean = h->d_bmean;
  a.ldata = h->svb_ldata;
  a.Cmom = P > 0 ? h->svb_cmom : nullptr;
  {
    Timed tm(h, BFMRI_T_ASSEMBLE_W);
    e = launch_assemble_w(a, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "svb assemble W");
  sv.scale = h->d_alpha;
  sv.spatial = 1;
  sv.vs = (size_t)K * ld;
  sv.rng = rng_of(h, counter, TAG_W);
  e = launch_svb(2, K, sv, h->stream, nullptr);
  if (e != cudaSuccess) return cuda_fail(h, e, "svb rhs W");
  MrhsArgs m = mrhs_args(h, K, S, h->d_alpha, h->opt.max_iter, false);
  mrhs_ssor(h, m);
  m.vs = (size_t)K * ld;
  m.x = h->svb_W;
  {
    Timed tm(h, BFMRI_T_PCG_W, true, 0);
    e = launch_mrhs(K, m, h->stream, nullptr);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "svb solve W");
  std::vector<RhsState> stW(S), stA;
  CU(h, cudaMemcpyAsync(stW.data(), h->mr_st, S * sizeof(RhsState), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  // ---- q(A): system averaged over the new W samples ----
  const double* bscale = spatial ? h->d_beta : h->d_zero;
  if (P > 0) {
    e = launch_svb(1, K, sv, h->stream, nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "svb gram");
    AssembleArgs b = assemble_args(h, bscale, 0, TAG_A);
    b.perturb = 0;
    b.blocks32 = nullptr;
    b.mfac32 = nullptr;
    b.bmean = h->d_bmean;
    b.ldata = h->svb_ldata;
    b.Gin = h->svb_gin;
    b.G = h->d_G;
    {
      Timed tm(h, BFMRI_T_ASSEMBLE_A);
      e = launch_assemble_a(b, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "svb assemble A");
    sv.scale = bscale;
    sv.spatial = spatial ? 1 : 0;
    sv.vs = (size_t)P * ld;
    sv.rng = rng_of(h, counter, TAG_A);
    e = launch_svb(2, P, sv, h->stream, nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "svb rhs A");
    MrhsArgs ma = mrhs_args(h, P, S, bscale, h->opt.max_iter, false);
    mrhs_ssor(h, ma);
    ma.vs = (size_t)P * ld;
    ma.x = h->svb_A;
    {
      Timed tm(h, BFMRI_T_PCG_A, true, 1);
      e = launch_mrhs(P, ma, h->stream, nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "svb solve A");
    stA.resize(S);
    CU(h, cudaMemcpyAsync(stA.data(), h->mr_st, S * sizeof(RhsState), cudaMemcpyDeviceToHost, h->stream));
  }
  // ---- q(lambda), then the quadratic forms for q(alpha), q(beta) ----
  {
    Timed tm(h, BFMRI_T_LAMBDA);
    e = launch_svb(3, K, sv, h->stream, nullptr);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "svb lambda");
  int grid = 0;
  e = launch_svb(4, K, sv, h->stream, &grid);
  if (e != cudaSuccess) return cuda_fail(h, e, "svb quad W");
  std::vector<double> partW((size_t)grid * K), partA;
  CU(h, cudaMemcpyAsync(partW.data(), h->svb_part, partW.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (P > 0 && spatial) {
    CU(h, cudaStreamSynchronize(h->stream));
    int gridA = 0;
    e = launch_svb(5, P, sv, h->stream, &gridA);
    if (e != cudaSuccess) return cuda_fail(h, e, "svb quad A");
    partA.resize((size_t)gridA * P);
    CU(h, cudaMemcpyAsync(partA.data(), h->svb_part, partA.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  RET(end_call(h, nullptr, nullptr));
  long long itW = 0, itA = 0;
  double worst = 0.0;
  for (const RhsState& r : stW) {
    if (r.status == 4) return fail(h, BFMRI_ERR_NOT_CONVERGED, "SVB W solve reached max_iter");
    if (r.status != 0) return fail(h, BFMRI_ERR_NOT_SPD, "SVB W solve breakdown");
    itW += r.total;
    worst = std::max(worst, r.bb > 0 ? std::sqrt(r.rr / r.bb) : 0.0);
  }
  for (const RhsState& r : stA) {
    if (r.status == 4) return fail(h, BFMRI_ERR_NOT_CONVERGED, "SVB A solve reached max_iter");
    if (r.status != 0) return fail(h, BFMRI_ERR_NOT_SPD, "SVB A solve breakdown");
    itA += r.total;
  }
  // E[alpha_k] = q~1k q~2, 1/q~1k = mean_j Q_k / 2 + 1/q1 (Eq. NFVB-alpha-parameters)
  auto hyper = [&](const std::vector<double>& part, int D, double r1, double r2, std::vector<double>& out) {
    const int g = (int)(part.size() / std::max(D, 1));
    out.assign(D, 0.0);
    for (int k = 0; k < D; ++k) {
      double q = 0.0;
      for (int b = 0; b < g; ++b) q += part[(size_t)b * D + k];
      q /= S;
      out[k] = (0.5 * h->N + r2) / (0.5 * q + 1.0 / r1);
    }
  };
  std::vector<double> avb, bvb;
  hyper(partW, K, h->opt.q1, h->opt.q2, avb);
  if (P > 0 && spatial) hyper(partA, P, h->opt.r1, h->opt.r2, bvb);
  if (alpha_vb) std::copy(avb.begin(), avb.end(), alpha_vb);
  if (beta_vb) std::copy(bvb.begin(), bvb.end(), beta_vb);
  // Appendix C, trick 1: every other iteration extrapolate from the last three values
  h->svb_iter += 1;
  bool extrapolated = false;
  auto trick = [&](std::vector<double>& vb, std::vector<double>* hist) -> std::vector<double> {
    std::vector<double> use = vb;
    if (extrapolate && h->svb_iter >= 3 && (h->svb_iter % 2) == 1 && hist[0].size() == vb.size() &&
        hist[1].size() == vb.size()) {
      for (size_t k = 0; k < vb.size(); ++k) {
        const double a2 = hist[0][k], a1 = hist[1][k], a0 = vb[k];
        const double c = 0.5 * (a2 - 2.0 * a1 + a0), d = 0.5 * (a2 - 4.0 * a1 + 3.0 * a0);
        double pred = (c != 0.0 && -d / (2.0 * c) > 0.0) ? a0 - d * d / (4.0 * c) : a1 + 20.0 * (a0 - a1);
        if (!(pred > 0.0)) pred = a0;
        use[k] = std::min(std::max(pred, a0 / 5.0), 5.0 * a0);
      }
      extrapolated = true;
    }
    hist[0] = hist[1];
    hist[1] = use;
    return use;
  };
  std::vector<double> au = trick(avb, h->svb_alpha_hist);
  CU(h, cudaMemcpyAsync(h->d_alpha, au.data(), K * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (P > 0 && spatial) {
    std::vector<double> bu = trick(bvb, h->svb_beta_hist);
    CU(h, cudaMemcpyAsync(h->d_beta, bu.data(), P * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  CU(h, cudaStreamSynchronize(h->stream));
  if (info) {
    info->iteration = h->svb_iter;
    info->samples = S;
    info->pcg_iterations_W = itW;
    info->pcg_iterations_A = itA;
    info->max_rel_residual_W = worst;
    info->extrapolated = extrapolated ? 1 : 0;
  }
  return BFMRI_OK;
}

bfmri_status bfmri_svb_get_sample(bfmri_handle* h, int j, double* W, double* A) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (j < 0 || j >= h->svb_S) return fail(h, BFMRI_ERR_INVALID_ARG, "no such SVB sample");
  if (W) RET(to_host(h, W, h->svb_W + (size_t)j * h->K * h->ld, h->K));
  if (A && h->P > 0) RET(to_host(h, A, h->svb_A + (size_t)j * h->P * h->ld, h->P));
  return BFMRI_OK;
}

bfmri_status bfmri_svb_set_sample(bfmri_handle* h, int j, const double* W, const double* A) {
  if (!h) return BFMRI_ERR_INVALID_ARG;
  if (j < 0 || j >= h->svb_S) return fail(h, BFMRI_ERR_INVALID_ARG, "no such SVB sample");
  if (W) RET(to_dev(h, h->svb_W + (size_t)j * h->K * h->ld, W, h->K));
  if (A && h->P > 0) RET(to_dev(h, h->svb_A + (size_t)j * h->P * h->ld, A, h->P));
  CU(h, cudaStreamSynchronize(h->stream));
  return BFMRI_OK;
}

bfmri_status bfmri_apply_precision(bfmri_handle* h, int which, const double* x, double* y) {
  RET(require_stats(h));
  if (!x || !y || (which != 0 && which != 1)) return fail(h, BFMRI_ERR_INVALID_ARG, "bad arguments");
  const int D = which == 0 ? h->K : h->P;
  if (D == 0) return BFMRI_OK;
  RET(begin_call(h));
  AssembleArgs a = assemble_args(h, which == 0 ? h->d_alpha : h->d_beta, 0, which == 0 ? TAG_W : TAG_A);
  a.perturb = 0;
  a.precond = 0;
  cudaError_t e = which == 0 ? launch_assemble_w(a, h->stream) : launch_assemble_a(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble");
  RET(to_dev(h, h->d_r, x, D));
  ApplyArgs ap;
  ap.g = geom(h);
  ap.D = D;
  ap.blocks = h->d_blocks;
  ap.scale = which == 0 ? h->d_alpha : h->d_beta;
  // the independent AR prior has no spatial term
  static const double zeros[PMAX] = {0, 0, 0, 0};
  if (which == 1 && h->opt.ar_prior != BFMRI_AR_SPATIAL) {
    CU(h, cudaMemcpyAsync(h->d_bmean, zeros, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    ap.scale = h->d_bmean;
  }
  ap.x = h->d_r;
  ap.y = h->d_z;
  ap.t = (which == 0 && h->opt.w_prior == BFMRI_PRIOR_LTL) ? h->d_lt : nullptr;
  ap.scale3 = (which == 0 && h->opt.w_prior == BFMRI_PRIOR_ANISO) ? h->d_alpha3 : nullptr;
  e = launch_apply(ap, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "apply");
  RET(end_call(h, nullptr, nullptr));
  return to_host(h, y, h->d_z, D);
}

bfmri_status bfmri_apply_preconditioner(bfmri_handle* h, int which, const double* x, double* y) {
  RET(require_stats(h));
  if (!x || !y || (which != 0 && which != 1)) return fail(h, BFMRI_ERR_INVALID_ARG, "bad arguments");
  const int D = which == 0 ? h->K : h->P;
  if (D == 0) return BFMRI_OK;
  if (which == 0 && h->opt.w_prior == BFMRI_PRIOR_ANISO && uses_ssor(h->opt))
    return fail(h, BFMRI_ERR_INVALID_ARG,
                "the anisotropic prior's reduced system has no separate preconditioner to inspect");
  if (h->d_ce && uses_ssor(h->opt))
    return fail(h, BFMRI_ERR_INVALID_ARG,
                "the reduced system with per-edge factors has no separate preconditioner to inspect");
  RET(begin_call(h));
  AssembleArgs a = assemble_args(h, which == 0 ? h->d_alpha : h->d_beta, 0, which == 0 ? TAG_W : TAG_A);
  a.perturb = 0;
  cudaError_t e = which == 0 ? launch_assemble_w(a, h->stream) : launch_assemble_a(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble");
  RET(to_dev(h, h->d_r, x, D));
  PcgArgs p;
  memset(&p, 0, sizeof(p));
  p.N = h->N;
  p.ld = h->ld;
  p.ndir = h->ndir;
  for (int d = 0; d < 3; ++d) p.cw[d] = h->opt.edge_weight[d];
  p.nbr = h->d_nbr;
  p.mfac = h->opt.precond != BFMRI_PRECOND_NONE ? h->d_mfac : nullptr;
  p.scale = which == 0 ? h->d_alpha : h->d_beta;
  // the independent AR prior has no spatial term
  static const double zeros[PMAX] = {0, 0, 0, 0};
  if (which == 1 && h->opt.ar_prior != BFMRI_AR_SPATIAL) {
    CU(h, cudaMemcpyAsync(h->d_bmean, zeros, D * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    p.scale = h->d_bmean;
  }
  p.r = h->d_r;
  p.u = h->d_z;
  p.ssor = uses_ssor(h->opt);
  p.omega = ssor_omega_of(h->opt);
  p.red = h->d_red;
  p.n_red = h->n_red;
  p.black = h->d_black;
  p.n_black = h->n_black;
  p.colour = h->d_colour;
  if (h->opt.precond == BFMRI_PRECOND_MULTIGRID) {
    RET(ensure_mg(h));
    MgArgs m = mg_args(h, p.scale, h->d_W, which);
    m.apply_only = 1;
    e = launch_mg_setup(D, m, h->stream);
    if (e == cudaSuccess) e = launch_pcg_mg(D, m, h->stream, nullptr);
  } else {
    e = launch_precond_apply(D, p, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "preconditioner apply");
  RET(end_call(h, nullptr, nullptr));
  return to_host(h, y, h->d_z, D);
}

bfmri_status bfmri_build_system(bfmri_handle* h, int which, uint64_t counter, double* blocks,
                                double* b_mean, double* b_pert) {
  RET(require_stats(h));
  if (which != 0 && which != 1) return fail(h, BFMRI_ERR_INVALID_ARG, "which must be 0 or 1");
  const int D = which == 0 ? h->K : h->P;
  if (D == 0) return BFMRI_OK;
  RET(begin_call(h));
  AssembleArgs a = assemble_args(h, which == 0 ? h->d_alpha : h->d_beta, counter, which == 0 ? TAG_W : TAG_A);
  a.precond = 0;
  a.bmean = h->d_bmean;
  cudaError_t e = cudaSuccess;
  if (a.ltl) e = launch_ltl_noise(a.g, h->K, h->d_alpha, a.rng, h->d_edge, h->stream);
  if (a.scale3) {
    e = launch_edge_noise(a.g, h->K, h->d_alpha, a.rng, h->d_edge, h->stream, a.scale3);
    a.edge = h->d_edge;
  }
  if (e == cudaSuccess) e = which == 0 ? launch_assemble_w(a, h->stream) : launch_assemble_a(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble");
  RET(end_call(h, nullptr, nullptr));
  if (blocks) {
    const int nt = ntri(D);
    std::vector<double> planes((size_t)nt * h->N);
    CU(h, cudaMemcpy2DAsync(planes.data(), (size_t)h->N * sizeof(double), h->d_blocks,
                            h->ld * sizeof(double), (size_t)h->N * sizeof(double), nt,
                            cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    for (int n = 0; n < h->N; ++n)
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          const int e2 = i >= j ? tri(i, j) : tri(j, i);
          blocks[((size_t)n * D + i) * D + j] = planes[(size_t)e2 * h->N + n];
        }
  }
  if (b_mean) RET(to_host(h, b_mean, h->d_bmean, D));
  if (b_pert) RET(to_host(h, b_pert, h->d_rhs, D));
  return BFMRI_OK;
}

}  // extern "C"
