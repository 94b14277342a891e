// PCG with the aggregation multigrid V-cycle preconditioner (mg.cuh), one cooperative launch
// per solve, FP64, vectors of every level in global memory, grid-stride loops over voxels.
//
// One PCG iteration (standard form, Hestenes & Stiefel, preconditioned):
//   q = B~ p, gamma = p'q                       --- reducing barrier ---
//   x += a p, r -= a q, z = M^-1 r (V-cycle, its own grid barriers), rho = r'z, rr = r'r
//                                               --- reducing barrier ---
//   p = z + (rho / rho_old) p                   --- barrier (q needs the neighbours' p) ---
// When the recursive residual reaches delta, the true residual b - B~ x confirms the stop or
// restarts the recurrence from it. All sums are fixed-order (grid_allreduce4).
#include "mg.cuh"

namespace bfmri {

namespace {

struct MgShared {
  double red[32 * 4 + 8];
  int ints[2];
  int flag;
};

template <int D>
__device__ __forceinline__ void load_vec(const double* V, size_t ld, int n, double* v) {
#pragma unroll
  for (int k = 0; k < D; ++k) v[k] = V[(size_t)k * ld + n];
}

template <int D>
__device__ __forceinline__ void store_vec(double* V, size_t ld, int n, const double* v) {
#pragma unroll
  for (int k = 0; k < D; ++k) V[(size_t)k * ld + n] = v[k];
}

// sum over the in-mask neighbours m of voxel n of w_nm V[m] (values written by other CTAs
// before the last grid barrier: read through L2)
template <int D>
__device__ __forceinline__ void wsum(const MgLevel& L, const double* V, int n, double* sum, double* deg) {
#pragma unroll
  for (int k = 0; k < D; ++k) sum[k] = 0.0;
  double dg = 0.0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int m = __ldg(L.nbr + (size_t)d * L.ld + n);
    if (m >= 0) {
      const double w = __ldg(L.wgt + (size_t)d * L.ld + n);
      dg += w;
#pragma unroll
      for (int k = 0; k < D; ++k) sum[k] += w * __ldcg(V + (size_t)k * L.ld + m);
    }
  }
  if (deg) *deg = dg;
}

// out = (L L')^-1 t with the level's Gauss-Seidel factor of voxel n
template <int D>
__device__ __forceinline__ void fac_solve(const MgLevel& L, int n, const double* t, double* out) {
  double F[ntri(D)];
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) F[e] = L.fac[(size_t)e * L.ld + n];
  chol_solve_invdiag<D>(F, t, out);
}

// out = A_l v at voxel n: blocks v + scale .* (deg v - sum_m w_nm V[m])
template <int D>
__device__ __forceinline__ void apply_level(const MgLevel& L, const double* s, const double* V, int n,
                                            const double* v, double* out) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) acc += __ldg(L.blocks + (size_t)(i >= j ? tri(i, j) : tri(j, i)) * L.ld + n) * v[j];
    out[i] = acc;
  }
  double sum[D], deg;
  wsum<D>(L, V, n, sum, &deg);
#pragma unroll
  for (int k = 0; k < D; ++k) out[k] += s[k] * (deg * v[k] - sum[k]);
}

}  // namespace

// Coarse blocks of level l (l >= 1): the sums of the children's blocks.
template <int D>
__global__ void k_mg_coarse_blocks(MgLevel fine, MgLevel coarse) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= coarse.N) return;
  double acc[ntri(D)];
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) acc[e] = 0.0;
  for (int j = 0; j < 8; ++j) {
    const int ch = coarse.child[(size_t)j * coarse.ld + c];
    if (ch < 0) continue;
#pragma unroll
    for (int e = 0; e < ntri(D); ++e) acc[e] += fine.blocks[(size_t)e * fine.ld + ch];
  }
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) const_cast<double*>(coarse.blocks)[(size_t)e * coarse.ld + c] = acc[e];
}

// Gauss-Seidel factor of level l (l >= 1): Cholesky of blocks + diag(scale) deg.
template <int D>
__global__ void k_mg_factor(MgLevel L, const double* scale, int* bad) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.N) return;
  double M[ntri(D)];
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) M[e] = L.blocks[(size_t)e * L.ld + c];
  double deg = 0.0;
  for (int d = 0; d < 6; ++d) deg += L.wgt[(size_t)d * L.ld + c];
#pragma unroll
  for (int k = 0; k < D; ++k) M[tri(k, k)] += __ldg(scale + k) * deg;
  if (!chol_packed_invdiag<D>(M)) atomicMin(bad, c);
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) L.fac[(size_t)e * L.ld + c] = M[e];
}

template <int D>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_mg(MgArgs a) {
  __shared__ MgShared sh;
  grid_barrier_start(a.bar);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  double s[D];
#pragma unroll
  for (int k = 0; k < D; ++k) s[k] = __ldg(a.scale + k);
  const MgLevel& F = a.lv[0];
  const size_t ld = F.ld;
  auto bar = [&]() -> bool { return grid_sync(a.bar, &sh.flag); };

  // level l, first half-sweep from x = 0: x = fac^-1 b at the red voxels, 0 at the black
  // ones. Voxels are taken in index order (the same thread owns voxel n as in the passes
  // that wrote b), so no barrier is needed before it.
  auto red_from_zero = [&](const MgLevel& L) {
    for (int n = tid; n < L.N; n += nth) {
      double t[D], x[D];
      if (__ldg(L.colour + n) == 0) {
        load_vec<D>(L.b, L.ld, n, t);
        fac_solve<D>(L, n, t, x);
      } else {
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = 0.0;
      }
      store_vec<D>(L.x, L.ld, n, x);
    }
  };
  // one colour's half-sweep: x_n = fac^-1 (b_n + scale .* sum_m w_nm x_m)
  auto half = [&](const MgLevel& L, const int* list, int cnt) {
    for (int i = tid; i < cnt; i += nth) {
      const int n = __ldg(list + i);
      double t[D], sum[D], x[D];
      load_vec<D>(L.b, L.ld, n, t);
      wsum<D>(L, L.x, n, sum, nullptr);
#pragma unroll
      for (int k = 0; k < D; ++k) t[k] += s[k] * sum[k];
      fac_solve<D>(L, n, t, x);
      store_vec<D>(L.x, L.ld, n, x);
    }
  };
  auto residual = [&](const MgLevel& L) {
    for (int n = tid; n < L.N; n += nth) {
      double xn[D], ax[D], b[D];
      load_vec<D>(L.x, L.ld, n, xn);
      load_vec<D>(L.b, L.ld, n, b);
      apply_level<D>(L, s, L.x, n, xn, ax);
#pragma unroll
      for (int k = 0; k < D; ++k) b[k] -= ax[k];
      store_vec<D>(L.r, L.ld, n, b);
    }
  };
  auto restrict_to = [&](const MgLevel& Lf, const MgLevel& Lc) {
    for (int c = tid; c < Lc.N; c += nth) {
      double acc[D];
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = 0.0;
      for (int j = 0; j < 8; ++j) {
        const int ch = __ldg(Lc.child + (size_t)j * Lc.ld + c);
        if (ch < 0) continue;
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] += __ldcg(Lf.r + (size_t)k * Lf.ld + ch);
      }
      store_vec<D>(Lc.b, Lc.ld, c, acc);
    }
  };
  auto prolong_from = [&](const MgLevel& Lf, const MgLevel& Lc) {
    for (int n = tid; n < Lf.N; n += nth) {
      const int c = __ldg(Lf.agg + n);
#pragma unroll
      for (int k = 0; k < D; ++k) Lf.x[(size_t)k * Lf.ld + n] += __ldcg(Lc.x + (size_t)k * Lc.ld + c);
    }
  };
  // z = M^-1 r: level 0's b is r and its x is z
  auto vcycle = [&]() -> bool {
    for (int l = 0; l + 1 < a.L; ++l) {
      const MgLevel& L = a.lv[l];
      red_from_zero(L);
      if (!bar()) return false;
      half(L, L.black, L.n_black);
      if (!bar()) return false;
      residual(L);
      if (!bar()) return false;
      restrict_to(L, a.lv[l + 1]);
      if (!bar()) return false;
    }
    const MgLevel& C = a.lv[a.L - 1];
    red_from_zero(C);
    for (int st = 0; st < a.coarse_steps; ++st) {
      if (!bar()) return false;
      half(C, C.black, C.n_black);
      if (!bar()) return false;
      half(C, C.red, C.n_red);
    }
    for (int l = a.L - 2; l >= 0; --l) {
      const MgLevel& L = a.lv[l];
      if (!bar()) return false;
      prolong_from(L, a.lv[l + 1]);
      if (!bar()) return false;
      half(L, L.black, L.n_black);
      if (!bar()) return false;
      half(L, L.red, L.n_red);
    }
    return bar();   // z is complete before any voxel-order pass reads it
  };
  double tot[4];
  auto allreduce = [&](const double* v) -> bool {
    return grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };

  if (a.apply_only) {
    vcycle();
    return;
  }
  // (re)start from the current x: r = b - B~ x, z = M^-1 r, p = z; partials r'z, r'r, b'b
  auto restart = [&](bool first) -> bool {
    if (!first && !bar()) return false;   // every x update is visible
    for (int n = tid; n < F.N; n += nth) {
      double xn[D], ax[D], b[D];
      load_vec<D>(a.x, ld, n, xn);
      load_vec<D>(a.b, ld, n, b);
      apply_level<D>(F, s, a.x, n, xn, ax);
#pragma unroll
      for (int k = 0; k < D; ++k) b[k] -= ax[k];
      store_vec<D>(a.r, ld, n, b);
    }
    if (!vcycle()) return false;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = tid; n < F.N; n += nth) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * ld + n;
        const double rk = a.r[o], zk = a.z[o], bk = __ldg(a.b + o);
        a.p[o] = zk;
        v[0] += rk * zk;
        v[2] += rk * rk;
        v[3] += bk * bk;
      }
    }
    return allreduce(v);
  };
  if (!restart(true)) return;
  const double bb = tot[3];
  const double tol2 = a.delta * a.delta * bb;
  const double rel0 = bb > 0.0 ? sqrt(tot[2] / bb) : 0.0;
  double rho = tot[0], rr = tot[2];
  int it = 0, restarts = 0, status = 0;
  if (!(isfinite(rho) && isfinite(bb))) status = 7;
  bool done = status != 0 || bb == 0.0 || rr <= tol2;
  if (status == 0 && bb == 0.0) {
    for (int n = tid; n < F.N; n += nth)
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = 0.0;
  }
  while (!done) {
    if (!bar()) return;                   // q = B~ p needs the neighbours' p
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = tid; n < F.N; n += nth) {
      double pn[D], qn[D];
      load_vec<D>(a.p, ld, n, pn);
      apply_level<D>(F, s, a.p, n, pn, qn);
      store_vec<D>(a.q, ld, n, qn);
#pragma unroll
      for (int k = 0; k < D; ++k) v[0] += pn[k] * qn[k];
    }
    if (!allreduce(v)) return;
    const double gam = tot[0];
    if (!(gam > 0.0) || !isfinite(gam)) {
      status = isfinite(gam) ? 3 : 7;
      break;
    }
    const double alpha = rho / gam;
    for (int n = tid; n < F.N; n += nth) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * ld + n;
        a.x[o] += alpha * a.p[o];
        a.r[o] -= alpha * a.q[o];
      }
    }
    ++it;
    if (!vcycle()) return;
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = tid; n < F.N; n += nth) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * ld + n;
        const double rk = a.r[o];
        w[0] += rk * a.z[o];
        w[2] += rk * rk;
      }
    }
    if (!allreduce(w)) return;
    const double rho_new = tot[0];
    rr = tot[2];
    if (!isfinite(rho_new) || !isfinite(rr)) {
      status = 7;
      break;
    }
    if (rr <= tol2 || it >= a.max_iter) {
      // confirm with the true residual (restart() recomputes r, z and p from x)
      if (!restart(false)) return;
      rr = tot[2];
      rho = tot[0];
      if (rr <= tol2) break;
      if (it >= a.max_iter) {
        status = 4;
        break;
      }
      ++restarts;
      continue;
    }
    const double beta = rho_new / rho;
    rho = rho_new;
    for (int n = tid; n < F.N; n += nth) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * ld + n;
        a.p[o] = a.z[o] + beta * a.p[o];
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->iterations = it;
    a.ctrl->restarts = restarts;
    a.ctrl->rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    a.ctrl->rel_res0 = rel0;
    a.ctrl->status = status;
    if (status != 0 && a.ctrl->status_any == 0) a.ctrl->status_any = status;
    a.ctrl->iter_total += it;
    a.ctrl->solves += 1;
  }
}

namespace {

template <int D>
cudaError_t mg_setup_d(const MgArgs& a, cudaStream_t s) {
  for (int l = 1; l < a.L; ++l) {
    const int g = (a.lv[l].N + 127) / 128;
    k_mg_coarse_blocks<D><<<g, 128, 0, s>>>(a.lv[l - 1], a.lv[l]);
    k_mg_factor<D><<<g, 128, 0, s>>>(a.lv[l], a.scale, a.bad_voxel);
  }
  return cudaGetLastError();
}

template <int D>
cudaError_t pcg_mg_d(const MgArgs& a, cudaStream_t stream, int* grid_out) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_mg<D>, PCG_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (a.sm_cap > 0 && a.sm_cap < nsm) nsm = a.sm_cap;
  int grid = nsm * per_sm;
  const int need = (a.lv[0].N + PCG_THREADS - 1) / PCG_THREADS;
  if (need < grid) grid = need < 1 ? 1 : need;
  if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
  if (grid_out) *grid_out = grid;
  e = reset_grid_barrier(a.bar, stream);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)k_pcg_mg<D>, dim3(grid), dim3(PCG_THREADS), args, 0, stream);
}

template <int D>
int mg_max_grid_d() {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_mg<D>, PCG_THREADS, 0);
  return nsm * (per_sm > 1 ? per_sm : 1);
}

}  // namespace

#define BFMRI_MG_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

cudaError_t launch_mg_setup(int D, const MgArgs& a, cudaStream_t stream) {
  switch (D) {
#define CASE(d) case d: return mg_setup_d<d>(a, stream);
    BFMRI_MG_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pcg_mg(int D, const MgArgs& a, cudaStream_t stream, int* grid_out) {
  switch (D) {
#define CASE(d) case d: return pcg_mg_d<d>(a, stream, grid_out);
    BFMRI_MG_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

int pcg_mg_max_grid(int D) {
  switch (D) {
#define CASE(d) case d: return mg_max_grid_d<d>();
    BFMRI_MG_CASES(CASE)
#undef CASE
    default: return 0;
  }
}

}  // namespace bfmri
