// Persistent, cooperative preconditioned conjugate gradients for the W and A draws
// (Algorithm 2, step 7: "solve B~ w = b approximately using PCG ... with starting value").
//
// One launch runs the whole solve. Each iteration is two grid-wide phases separated by a
// bounded grid barrier:
//   phase 1: p = z + beta p_prev (for the voxel and, on the fly, for its neighbours, so that
//            no third barrier is needed), q = B~ p (per-voxel block + stencil), partial p'q;
//   phase 2: x += a p, r -= a q, z = M^-1 r (block-Jacobi), partials r'z and r'r.
// The stop test uses the recursive residual and is confirmed with the true residual
// b - B~ x in FP64 (the paper's relative-residual criterion, Section 3.1); if the true
// residual is above tolerance the iteration restarts from it. All reductions are
// deterministic (fixed-order), so a solve is bit-reproducible run to run.
#include "pcg.cuh"

namespace bfmri {

namespace {

// Data written by other CTAs during the launch must bypass L1 (not coherent across SMs).
__device__ __forceinline__ double ldx(const double* p) { return __ldcg(p); }

template <int D>
struct Vox {
  // Applies the stencil part: out += s .* (deg * pn - sum_m pm), with pm supplied by f(m, k).
  template <typename F>
  __device__ __forceinline__ static void stencil(const PcgArgs& a, int n, const double* s,
                                                 const double* pn, double* out, F f) {
    double sum[D];
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] = 0.0;
    int deg = 0;
    for (int d = 0; d < a.ndir; ++d) {
      const int m = __ldg(a.nbr + (size_t)d * a.ld + n);
      if (m >= 0) {
        ++deg;
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += f(m, k);
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) out[k] += s[k] * ((double)deg * pn[k] - sum[k]);
  }
};

template <int D>
__device__ __forceinline__ void block_mul(const PcgArgs& a, int n, const double* p, double* q) {
  double B[ntri(D)];
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) B[e] = __ldg(a.blocks + (size_t)e * a.ld + n);
  sym_mul<D>(B, p, q);
}

template <int D>
__device__ __forceinline__ void precond(const PcgArgs& a, int n, const double* r, double* z) {
  if (a.mfac == nullptr) {
#pragma unroll
    for (int k = 0; k < D; ++k) z[k] = r[k];
    return;
  }
  double L[ntri(D)];
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) L[e] = __ldg(a.mfac + (size_t)e * a.ld + n);
  chol_solve_invdiag<D>(L, r, z);
}

// r = b - B~ x for voxel n (x of neighbours read through L2); returns it in rn.
template <int D>
__device__ __forceinline__ void true_residual(const PcgArgs& a, int n, const double* s, double* rn) {
  double xn[D], Ax[D];
#pragma unroll
  for (int k = 0; k < D; ++k) xn[k] = ldx(a.x + (size_t)k * a.ld + n);
  block_mul<D>(a, n, xn, Ax);
  Vox<D>::stencil(a, n, s, xn, Ax, [&](int m, int k) { return ldx(a.x + (size_t)k * a.ld + m); });
#pragma unroll
  for (int k = 0; k < D; ++k) rn[k] = __ldg(a.b + (size_t)k * a.ld + n) - Ax[k];
}

}  // namespace

template <int D>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg(PcgArgs a) {
  __shared__ double sh_red[32 * 4];
  __shared__ double sh_tot[4];
  __shared__ int sh_flag;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const size_t ld = a.ld;
  double s[D];
#pragma unroll
  for (int k = 0; k < D; ++k) s[k] = __ldg(a.scale + k);
  const double delta = a.delta;
  const int max_iter = a.max_iter;
  double* part[2] = {a.part, a.part + (size_t)gridDim.x * 4};
  int pb = 0;  // partial buffer toggle

  auto sync = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;   // test hook: never arrive
    return grid_sync(a.bar, &sh_flag);
  };

  // ---- setup: r = b - B~ x, z = M^-1 r ----
  {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = tid; n < a.N; n += nth) {
      double rn[D], zn[D];
      true_residual<D>(a, n, s, rn);
      precond<D>(a, n, rn, zn);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a.r[k * ld + n] = rn[k];
        a.z[k * ld + n] = zn[k];
        const double bk = __ldg(a.b + (size_t)k * ld + n);
        acc[0] += rn[k] * zn[k];
        acc[1] += rn[k] * rn[k];
        acc[2] += bk * bk;
      }
    }
    block_partial<4>(acc, sh_red, part[pb]);
  }
  if (!sync()) return;
  double tot[4];
  grid_total<4>(part[pb], sh_tot, tot);
  pb ^= 1;
  double rho = tot[0], rr = tot[1];
  const double bb = tot[2];
  const double tol2 = delta * delta * bb;
  int it = 0, restarts = 0, status = 0;
  const bool finite0 = isfinite(rho) && isfinite(rr) && isfinite(bb);
  if (!finite0) status = 7;
  if (bb == 0.0 && status == 0) {
    // B~ is SPD, so the solution of B~ x = 0 is x = 0.
    for (int n = tid; n < a.N; n += nth)
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[k * ld + n] = 0.0;
  }
  const double rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  bool done = (status != 0) || bb == 0.0 || rr <= tol2;
  double rr_final = rr;
  bool first = true;
  double beta = 0.0;
  double* pprev = a.p0;
  double* pnext = a.p1;

  while (!done) {
    // ---- phase 1: p = z + beta p_prev ; q = B~ p ; p'q ----
    {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int n = tid; n < a.N; n += nth) {
        double pn[D], qn[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double zk = ldx(a.z + (size_t)k * ld + n);
          pn[k] = first ? zk : zk + beta * ldx(pprev + (size_t)k * ld + n);
        }
        block_mul<D>(a, n, pn, qn);
        Vox<D>::stencil(a, n, s, pn, qn, [&](int m, int k) {
          const double zm = ldx(a.z + (size_t)k * ld + m);
          return first ? zm : zm + beta * ldx(pprev + (size_t)k * ld + m);
        });
#pragma unroll
        for (int k = 0; k < D; ++k) {
          pnext[k * ld + n] = pn[k];
          a.q[k * ld + n] = qn[k];
          acc[0] += pn[k] * qn[k];
        }
      }
      block_partial<4>(acc, sh_red, part[pb]);
    }
    if (!sync()) return;
    grid_total<4>(part[pb], sh_tot, tot);
    pb ^= 1;
    const double gam = tot[0];
    if (!(gam > 0.0) || !isfinite(gam)) { status = isfinite(gam) ? 3 : 7; break; }
    const double alpha = rho / gam;
    // ---- phase 2: x += alpha p ; r -= alpha q ; z = M^-1 r ; r'z, r'r ----
    {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int n = tid; n < a.N; n += nth) {
        double rn[D], zn[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double pk = pnext[k * ld + n];
          const double qk = a.q[k * ld + n];
          a.x[k * ld + n] += alpha * pk;
          rn[k] = a.r[k * ld + n] - alpha * qk;
          a.r[k * ld + n] = rn[k];
        }
        precond<D>(a, n, rn, zn);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          a.z[k * ld + n] = zn[k];
          acc[0] += rn[k] * zn[k];
          acc[1] += rn[k] * rn[k];
        }
      }
      block_partial<4>(acc, sh_red, part[pb]);
    }
    if (!sync()) return;
    grid_total<4>(part[pb], sh_tot, tot);
    pb ^= 1;
    ++it;
    const double rho_new = tot[0];
    rr = tot[1];
    if (!isfinite(rho_new) || !isfinite(rr)) { status = 7; break; }
    {
      double* t = pprev; pprev = pnext; pnext = t;
    }
    if (rr <= tol2 || it >= max_iter) {
      // ---- confirm with the true residual (paper: ||B~ x - b|| / ||b|| < delta) ----
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int n = tid; n < a.N; n += nth) {
        double rn[D], zn[D];
        true_residual<D>(a, n, s, rn);
        precond<D>(a, n, rn, zn);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          a.r[k * ld + n] = rn[k];
          a.z[k * ld + n] = zn[k];
          acc[0] += rn[k] * zn[k];
          acc[1] += rn[k] * rn[k];
        }
      }
      block_partial<4>(acc, sh_red, part[pb]);
      if (!sync()) return;
      grid_total<4>(part[pb], sh_tot, tot);
      pb ^= 1;
      rr_final = tot[1];
      if (rr_final <= tol2) break;
      if (it >= max_iter) { status = 4; break; }
      ++restarts;
      rho = tot[0];
      first = true;
      continue;
    }
    beta = rho_new / rho;
    rho = rho_new;
    first = false;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->iterations = it;
    a.ctrl->restarts = restarts;
    a.ctrl->rel_res = bb > 0.0 ? sqrt((status == 0 ? rr_final : rr) / bb) : 0.0;
    a.ctrl->rel_res0 = rel0;
    a.ctrl->status = status;
    if (status != 0 && a.ctrl->status_any == 0) a.ctrl->status_any = status;
    a.ctrl->iter_total += it;
    a.ctrl->solves += 1;
  }
}

template <int D>
static cudaError_t launch_d(const PcgArgs& a, cudaStream_t stream, int* grid_out) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<D>, PCG_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int need = (a.N + PCG_THREADS - 1) / PCG_THREADS;
  int grid = nsm * per_sm;
  if (need < grid) grid = need < 1 ? 1 : need;
  if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
  if (grid_out) *grid_out = grid;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)k_pcg<D>, dim3(grid), dim3(PCG_THREADS), args, 0, stream);
}

template <int D>
static int max_grid_d() {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<D>, PCG_THREADS, 0);
  return nsm * per_sm;
}

#define BFMRI_PCG_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

cudaError_t launch_pcg(int D, const PcgArgs& a, cudaStream_t stream, int* grid_out) {
  switch (D) {
#define CASE(d) case d: return launch_d<d>(a, stream, grid_out);
    BFMRI_PCG_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

int pcg_max_grid(int D) {
  switch (D) {
#define CASE(d) case d: return max_grid_d<d>();
    BFMRI_PCG_CASES(CASE)
#undef CASE
    default: return 0;
  }
}

}  // namespace bfmri
