// Multi-right-hand-side PCG (one matrix, S right-hand sides) in one cooperative launch.
// Used by the log-determinant / trace probes and by the spatial-VB step, whose N_s samples
// all solve with the one matrix B~_SVB and so can share its preconditioner (Section 3.3).
//
// Work decomposition: the grid's warps are split into S x C units (right-hand side r, voxel
// chunk c); lanes of a warp take consecutive voxels of the chunk, so every vector access is
// coalesced, and each unit produces one row of partial sums. At each reducing barrier the CTA
// that arrives last sums the rows of every right-hand side in a fixed order and advances its
// CG scalars (Chronopoulos-Gear recurrence, as in the single solve), records the CG
// coefficients (alpha_j, beta_j) of the first run for Lanczos quadrature, and marks converged
// right-hand sides, which then stop moving. Converged right-hand sides are confirmed with the
// true residual b - B~ x before they are released.
#pragma once
// The multi-RHS solver kernels and their launchers, included by the translation units that
// instantiate them for groups of D (kernels_mrhs_d*.cu); kernels_mrhs.cu holds the dispatch
// by D and the probe kernels.
#include "mrhs.cuh"

namespace bfmri {

namespace {

constexpr int MRHS_THREADS = 256;

// out = B v + s .* (deg v - sum of the neighbours' V), for voxel n.
// All neighbour indices are loaded first and then all neighbour values, so that one group of
// loads is in flight instead of a chain of dependent index -> value round trips (an absent
// neighbour reads the voxel's own value, which is masked out). FP64 solves take the six
// directions in two halves to bound the registers held.
// Neighbour values go through L1: lanes of a warp share the lines of their +-x and +-y
// neighbours. They were written by other CTAs before the last grid barrier, whose gpu-scope
// acquire orders these loads after those writes.
struct Units {
  int S, chunks, units, csize, gw, nw, lane;
  const int* first = nullptr;   // uneven masks: right-hand side r owns units first[r] .. first[r + 1] - 1
};

__device__ __forceinline__ Units units_of(const MrhsArgs& a) {
  Units u;
  u.S = a.S;
  u.nw = (gridDim.x * blockDim.x) >> 5;
  u.gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  u.lane = threadIdx.x & 31;
  u.chunks = u.nw / a.S;
  if (u.chunks < 1) u.chunks = 1;
  u.units = a.S * u.chunks;
  int cs = (a.N + u.chunks - 1) / u.chunks;
  u.csize = ((cs + 31) / 32) * 32;
  u.first = nullptr;
  return u;
}

// Work units: without uneven masks every right-hand side has U.chunks units and unit
// c S + r is chunk c of right-hand side r; with them right-hand side r has the units
// first[r] .. first[r + 1] - 1, as many as its share of the voxels. Unit u writes partial
// row u either way.
__device__ __forceinline__ int unit_count(const Units& U, int r) {
  return U.first ? U.first[r + 1] - U.first[r] : U.chunks;
}
__device__ __forceinline__ int unit_row(const Units& U, int r, int c) {
  return U.first ? U.first[r] + c : c * U.S + r;
}
__device__ __forceinline__ int unit_rhs_of(const Units& U, int u) {
  if (!U.first) return u % U.S;
  int lo = 0, hi = U.S - 1;   // the last r with first[r] <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (U.first[mid] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int unit_chunk_of(const Units& U, int u) {
  return U.first ? u - U.first[unit_rhs_of(U, u)] : u / U.S;
}

// Operator, scales, b and x of right-hand side r, and the lattice it lives on (its own with
// uneven masks, else the launch's): voxels, plane stride, neighbour planes, colour lists, edge
// weights, and its voxel chunks (nch chunks of cs voxels).
template <int D, typename T>
struct RhsOp {
  const T* B;
  const T* M;
  const T* b;
  T* x;
  T sc[D];
  int N, ndir, n_red, n_black, nch, cs;
  size_t ld;
  const int* nbr;
  const int* red;
  const int* black;
  T cw[3];
};

template <int D, typename T>
__device__ __forceinline__ RhsOp<D, T> rhs_op(const MrhsArgs& a, const Units& U, int r) {
  RhsOp<D, T> o;
  const double* scale;
  if (a.tab != nullptr) {
    const MrhsRhsPtrs& t = a.tab[r];
    o.B = static_cast<const T*>(t.blocks);
    o.M = static_cast<const T*>(t.mfac);
    o.b = static_cast<const T*>(t.b);
    o.x = static_cast<T*>(t.x);
    scale = t.scale;
  } else {
    o.B = static_cast<const T*>(a.blocks);
    o.M = static_cast<const T*>(a.mfac);
    o.b = static_cast<const T*>(a.b) + (size_t)r * a.vs;
    o.x = static_cast<T*>(a.x) + (size_t)r * a.vs;
    scale = a.scale;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) o.sc[k] = (T)__ldg(scale + k);
  if (a.uneven) {
    const MrhsRhsPtrs& t = a.tab[r];
    o.N = t.N;
    o.ndir = t.ndir;
    o.ld = t.ld;
    o.nbr = t.nbr;
    o.red = t.red;
    o.black = t.black;
    o.n_red = t.n_red;
    o.n_black = t.n_black;
#pragma unroll
    for (int d = 0; d < 3; ++d) o.cw[d] = (T)t.cw[d];
  } else {
    o.N = a.N;
    o.ndir = a.ndir;
    o.ld = a.ld;
    o.nbr = a.nbr;
    o.red = a.red;
    o.black = a.black;
    o.n_red = a.n_red;
    o.n_black = a.n_black;
#pragma unroll
    for (int d = 0; d < 3; ++d) o.cw[d] = (T)a.cw[d];
  }
  o.nch = unit_count(U, r);
  const int cs = (o.N + o.nch - 1) / o.nch;
  o.cs = ((cs + 31) / 32) * 32;
  return o;
}

// out = B v + s .* (deg v - sum of the neighbours' V), for voxel n of right-hand side op.
// All neighbour indices are loaded first and then all neighbour values, so that one group of
// loads is in flight instead of a chain of dependent index -> value round trips (an absent
// neighbour reads the voxel's own value, which is masked out). FP64 solves take the six
// directions in two halves to bound the registers held.
// Neighbour values go through L1: lanes of a warp share the lines of their +-x and +-y
// neighbours. They were written by other CTAs before the last grid barrier, whose gpu-scope
// acquire orders these loads after those writes.
template <int D, typename T>
__device__ __forceinline__ void block_apply(const RhsOp<D, T>& op, int n, const T* v, const T* V, T* out) {
  const size_t ld = op.ld;
  int nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = d < op.ndir ? __ldg(op.nbr + (size_t)d * ld + n) : -1;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) acc += __ldg(op.B + (size_t)(i >= j ? tri(i, j) : tri(j, i)) * ld + n) * v[j];
    out[i] = acc;
  }
  T sum[D];
#pragma unroll
  for (int k = 0; k < D; ++k) sum[k] = T(0);
  T deg = T(0);
  constexpr int H = sizeof(T) == 4 ? 6 : 3;   // directions per round of loads
#pragma unroll
  for (int d0 = 0; d0 < 6; d0 += H) {
    T nv[H][D];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int m = nb[d0 + h] >= 0 ? nb[d0 + h] : n;
#pragma unroll
      for (int k = 0; k < D; ++k) nv[h][k] = V[(size_t)k * ld + m];
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
      if (nb[d0 + h] >= 0) {
        const T c = op.cw[(d0 + h) >> 1];   // edge weight of the slot's direction
        deg += c;
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += c * nv[h][k];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) out[k] += op.sc[k] * (deg * v[k] - sum[k]);
}

// Compensated (Kahan) accumulation in the storage type: per-thread partial sums stay
// accurate without a per-voxel FP64 operation (FP64 issue is scarce on this part); each
// work unit converts its sums to FP64 once.
template <typename T>
struct KSum {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// FP64 partial sums need no compensation: plain accumulation (one FP64 add per term).
template <>
struct KSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

template <int D, typename T>
__device__ __forceinline__ void precond_apply(const RhsOp<D, T>& op, int n, const T* r, T* z) {
  if (op.M == nullptr) {
#pragma unroll
    for (int k = 0; k < D; ++k) z[k] = r[k];
    return;
  }
  T L[ntri(D)];
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) L[e] = __ldg(op.M + (size_t)e * op.ld + n);
  chol_solve_invdiag<D>(L, r, z);
}

// RHS state written by whichever CTA completed an earlier reduction: read through L2.
__device__ __forceinline__ RhsState load_state(const RhsState* p) {
  RhsState s;
  s.gam = __ldcg(&p->gam);
  s.alpha = __ldcg(&p->alpha);
  s.beta = __ldcg(&p->beta);
  s.bb = __ldcg(&p->bb);
  s.rr = __ldcg(&p->rr);
  s.rr0 = __ldcg(&p->rr0);
  s.active = __ldcg(&p->active);
  s.iters = __ldcg(&p->iters);
  s.total = __ldcg(&p->total);
  s.restarts = __ldcg(&p->restarts);
  s.hist_ok = __ldcg(&p->hist_ok);
  s.status = __ldcg(&p->status);
  return s;
}

// mode 0: (re)start pass for right-hand sides in phase 1 (pending check) or all (first pass);
// mode 1: iteration pass for active right-hand sides.
// Scalar logic run by the last CTA; returns (through flags[0]) whether any RHS is active.
__device__ __forceinline__ void scalar_logic(const MrhsArgs& a, int r, const double* t, int mode, bool first) {
  RhsState st = load_state(a.st + r);
  const double tol2 = a.delta * a.delta * (first ? t[3] : st.bb);
  if (mode == 0) {
    if (first) {
      st.bb = t[3];
      st.rr0 = t[2];
      st.iters = 0;
      st.total = 0;
      st.restarts = 0;
      st.hist_ok = 1;
      st.status = 0;
      st.active = 1;
    }
    if (!(st.active == 1 || st.active == 2)) {  // already done
      a.st[r] = st;
      return;
    }
    st.rr = t[2];
    if (!(isfinite(t[0]) && isfinite(t[1]) && isfinite(t[2]))) {
      st.status = 7;
      st.active = 0;
    } else if (st.bb == 0.0 || t[2] <= tol2) {
      st.active = 0;                      // confirmed
    } else if (st.total >= a.max_iter || st.restarts > a.max_restarts) {
      st.status = 4;
      st.active = 0;
    } else {
      if (!first) {
        st.restarts += 1;
        st.hist_ok = 0;
      }
      st.gam = t[0];
      st.alpha = t[1] > 0.0 ? t[0] / t[1] : 0.0;
      st.beta = 0.0;
      st.active = t[1] > 0.0 ? 1 : 0;
      if (!(t[1] > 0.0)) st.status = 3;
    }
  } else {
    if (st.active != 1) {
      a.st[r] = st;
      return;
    }
    const double gnew = t[0], dnew = t[1];
    st.rr = t[2];
    st.total += 1;
    if (st.hist_ok) st.iters += 1;
    if (!(isfinite(gnew) && isfinite(dnew) && isfinite(st.rr))) {
      st.status = 7;
      st.active = 0;
      a.st[r] = st;
      return;
    }
    const double beta = gnew / st.gam;
    if (a.hist && st.hist_ok && st.iters <= a.hist_len) {
      a.hist[((size_t)(st.iters - 1) * a.S + r) * 2 + 0] = st.alpha;
      a.hist[((size_t)(st.iters - 1) * a.S + r) * 2 + 1] = beta;
    }
    if (st.rr <= tol2 || st.total >= a.max_iter) {
      st.active = 2;                      // pending confirmation by the true residual
    } else {
      const double den = dnew - beta * gnew / st.alpha;
      if (!(den > 0.0)) {
        st.status = 3;
        st.active = 0;
      } else {
        st.beta = beta;
        st.alpha = gnew / den;
        st.gam = gnew;
      }
    }
  }
  a.st[r] = st;
}

// Reducing barrier: per-unit partials -> per-RHS totals -> scalar logic (last CTA).
// Returns false on barrier failure; *any_active / *any_pending report the RHS states.
__device__ __forceinline__ bool mrhs_reduce(const MrhsArgs& a, const Units& U, int mode, bool first,
                                            int* sh_int, int* any_active, int* any_pending) {
  __syncthreads();
  if (threadIdx.x == 0) {
    // the arrival counter only grows during a launch: the last CTA of barrier g0 is the one
    // whose arrival takes it to (g0 + 1) x gridDim.x
    const unsigned int g0 = g_bar_gen;
    const unsigned int arrived = atom_add_acq_rel(a.bar.count, 1u);
    sh_int[0] = (arrived == (g0 + 1u) * gridDim.x - 1u) ? 1 : 0;
    sh_int[1] = (int)g0;
    sh_int[2] = 0;
    sh_int[3] = 0;
  }
  __syncthreads();
  if (sh_int[0]) {
    const int warp = threadIdx.x >> 5, nwc = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < a.S; r += nwc) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      const int nc = unit_count(U, r);
      for (int c = lane; c < nc; c += 32) {
        const size_t row = (size_t)unit_row(U, r, c);
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += __ldcg(a.part + row * 4 + i);
      }
      const double v = warp_reduce4(acc);
      double t[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) t[i] = __shfl_sync(0xffffffffu, v, 8 * i);
      if (lane == 0) {
        scalar_logic(a, r, t, mode, first);
        const int act = __ldcg(&a.st[r].active);
        if (act == 1) atomicOr(&sh_int[2], 1);
        if (act == 2) atomicOr(&sh_int[3], 1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.flags[0] = sh_int[2];
      a.flags[1] = sh_int[3];
      __threadfence();
      st_release(a.bar.gen, (unsigned int)sh_int[1] + 1u);
      g_bar_gen = (unsigned int)sh_int[1] + 1u;
    }
    __syncthreads();
  } else {
    if (threadIdx.x == 0) {
      const bool ok = wait_reach(a.bar, a.bar.gen, (unsigned int)sh_int[1] + 1u);
      g_bar_gen = (unsigned int)sh_int[1] + 1u;
      sh_int[2] = ok ? __ldcg(a.flags + 0) : 0;
      sh_int[3] = ok ? __ldcg(a.flags + 1) : 0;
      sh_int[0] = ok ? 0 : 1;
    }
    __syncthreads();
    if (sh_int[0]) return false;
  }
  *any_active = sh_int[2];
  *any_pending = sh_int[3];
  __syncthreads();
  return true;
}

}  // namespace

// FP32 solves stage their vector streams through shared memory (cp.async); FP64 solves,
// whose stages would not fit twice per SM, load directly.
template <typename T>
constexpr bool kStaged = sizeof(T) == 4;

template <int D, typename T>
constexpr size_t mrhs_stage_bytes() {
  return kStaged<T> ? (size_t)(MRHS_THREADS / 32) * 2 * (6 * D) * 32 * sizeof(T) : 0;
}

// FP32 solves and small FP64 systems run two CTAs per SM; FP64 systems with D > 4 take the
// whole register file of one CTA per SM, which removes their register spills.
template <int D, typename T>
__global__ void __launch_bounds__(MRHS_THREADS, (sizeof(T) == 4 || D <= 4) ? 2 : 1) k_mrhs(MrhsArgs a) {
  extern __shared__ __align__(16) unsigned char mrhs_smem[];
  T* stage = reinterpret_cast<T*>(mrhs_smem);
  T* Rv = static_cast<T*>(a.r);
  T* UUv = static_cast<T*>(a.u);
  T* WWv = static_cast<T*>(a.w);
  T* PPv = static_cast<T*>(a.p);
  T* SSv = static_cast<T*>(a.s);
  __shared__ int sh_int[4];
  __shared__ int sh_flag;
  Units U = units_of(a);
  grid_barrier_start(a.bar);
  __shared__ int sh_first[MRHS_UNEVEN_MAX_S + 1];
  if (a.uneven) {
    // every CTA derives the same unit ranges: one unit per right-hand side, and the warps
    // beyond those shared in proportion to the right-hand sides' voxels
    if (threadIdx.x == 0) {
      long long tot = 0;
      for (int r = 0; r < a.S; ++r) tot += a.tab[r].N;
      const long long extra = U.nw > a.S ? U.nw - a.S : 0;
      int acc = 0;
      for (int r = 0; r < a.S; ++r) {
        sh_first[r] = acc;
        acc += 1 + (tot > 0 ? (int)(extra * a.tab[r].N / tot) : 0);
      }
      sh_first[a.S] = acc;
    }
    __syncthreads();
    U.first = sh_first;
    U.units = sh_first[a.S];
  }
  auto unit_rhs = [&](int u) { return unit_rhs_of(U, u); };
  auto unit_chunk = [&](int u) { return unit_chunk_of(U, u); };
  // columns selected by `cols` (bit j = column j) of unit u's partial row
  auto write_partials = [&](int u, double* acc, unsigned cols) {
    const double v = warp_reduce4(acc);
    if ((U.lane & 7) == 0 && ((cols >> (U.lane >> 3)) & 1u)) a.part[(size_t)u * 4 + (U.lane >> 3)] = v;
  };
  // mode-0 pass: r = b - B~ x, u = M^-1 r, publish u; then w = B~ u and partials
  // for every RHS selected by `sel` (state 1 on the first pass, 2 afterwards).
  // SSOR phases 2 (black voxels) and 3 (red voxels) of every right-hand side selected by
  // `sel(r)`, each after a grid barrier: units (rhs, chunk of the colour list), lanes over
  // consecutive list entries. u holds z in place (see the single-solve kernels):
  //   black n: u_n = (2 - omega) omega Dg_n^-1 (r_n + scale .* sum_m u_m)
  //   red n:   u_n = (2 - omega) u_n + omega Dg_n^-1 (scale .* sum_m u_m)
  auto ssor_phases = [&](auto sel) -> bool {
    const T omega = (T)a.omega, c2 = T(2) - omega;
    for (int phase = 2; phase <= 3; ++phase) {
      if (!grid_sync(a.bar, &sh_flag)) return false;
      for (int u = U.gw; u < U.units; u += U.nw) {
        const int r = unit_rhs(u), c = unit_chunk(u);
        if (!sel(r)) continue;
        const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
        const int* list = phase == 2 ? op.black : op.red;
        const int nl = phase == 2 ? op.n_black : op.n_red;
        int cs = (nl + op.nch - 1) / op.nch;
        cs = ((cs + 31) / 32) * 32;
        const T* R = Rv + (size_t)r * a.vs;
        T* Uu = UUv + (size_t)r * a.vs;
        const int i1 = min(nl, (c + 1) * cs);
        for (int i = c * cs + U.lane; i < i1; i += 32) {
          const int n = __ldg(list + i);
          int nb[6];
#pragma unroll
          for (int d = 0; d < 6; ++d) nb[d] = d < op.ndir ? __ldg(op.nbr + (size_t)d * ld + n) : -1;
          T sum[D];
#pragma unroll
          for (int k = 0; k < D; ++k) sum[k] = T(0);
#pragma unroll
          for (int d = 0; d < 6; ++d) {
            if (nb[d] >= 0) {
#pragma unroll
              for (int k = 0; k < D; ++k) sum[k] += op.cw[d >> 1] * Uu[(size_t)k * ld + nb[d]];
            }
          }
          T t[D], z[D];
#pragma unroll
          for (int k = 0; k < D; ++k) t[k] = phase == 2 ? R[(size_t)k * ld + n] + op.sc[k] * sum[k] : op.sc[k] * sum[k];
          precond_apply<D, T>(op, n, t, z);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const size_t o = (size_t)k * ld + n;
            Uu[o] = phase == 2 ? c2 * omega * z[k] : c2 * Uu[o] + omega * z[k];
          }
        }
      }
    }
    return true;
  };
  // ---- red-black reduced system (a.reduced): CG on the black voxels' Schur complement
  // S = Dg_b - L Dg_r^-1 U preconditioned by Dg_b (the iterates of SSOR with omega = 1); the
  // red voxels' x is recovered from their own rows at every (re)start. u lives at the black
  // voxels of the U planes and y = Dg_r^-1 (scale .* sum of the black neighbours' u) at the
  // red ones; every warp owns at most one unit (the launcher guarantees S <= warps).
  auto list_chunk = [&](const RhsOp<D, T>& op, int nl, int c, int& i0, int& i1) {
    int cs = (nl + op.nch - 1) / op.nch;
    cs = ((cs + 31) / 32) * 32;
    i0 = c * cs;
    i1 = min(nl, (c + 1) * cs);
  };
  // sum over the in-mask neighbours m of V[m]
  auto nsum = [&](const RhsOp<D, T>& op, int n, const T* V, T* out) {
    const size_t ld = op.ld;
    int nb[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = d < op.ndir ? __ldg(op.nbr + (size_t)d * ld + n) : -1;
    T v[6][D];
#pragma unroll
    for (int d = 0; d < 6; ++d)
#pragma unroll
      for (int k = 0; k < D; ++k) v[d][k] = V[(size_t)k * ld + (nb[d] >= 0 ? nb[d] : n)];
#pragma unroll
    for (int k = 0; k < D; ++k) out[k] = T(0);
#pragma unroll
    for (int d = 0; d < 6; ++d)
      if (nb[d] >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) out[k] += op.cw[d >> 1] * v[d][k];
      }
  };
  // red voxels of the selected right-hand sides: U = Dg^-1 (scale .* sum of the neighbours' U)
  auto rb_red_phase = [&](auto sel) {
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int r = unit_rhs(u), c = unit_chunk(u);
      if (!sel(r)) continue;
      const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
      T* Uu = UUv + (size_t)r * a.vs;
      int i0, i1;
      list_chunk(op, op.n_red, c, i0, i1);
      for (int i = i0 + U.lane; i < i1; i += 32) {
        const int n = __ldg(op.red + i);
        T t[D], z[D];
        nsum(op, n, Uu, t);
#pragma unroll
        for (int k = 0; k < D; ++k) t[k] *= op.sc[k];
        precond_apply<D, T>(op, n, t, z);
#pragma unroll
        for (int k = 0; k < D; ++k) Uu[(size_t)k * ld + n] = z[k];
      }
    }
  };
  // (re)start: red x from its rows, black r = b - B~ x (the rows' true residual), u, w = S u;
  // partials (r'u, w'u, ||b - B~ x||^2 over every voxel, ||b||^2)
  auto restart_pass_rb = [&](bool first) -> bool {
    auto sel = [&](int r) { return first || __ldcg(&a.st[r].active) == 2; };
    KSum<T> kg, kd, krr, kbb;
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int r = unit_rhs(u), c = unit_chunk(u);
      if (!sel(r)) continue;
      const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
      int i0, i1;
      list_chunk(op, op.n_red, c, i0, i1);
      for (int i = i0 + U.lane; i < i1; i += 32) {
        const int n = __ldg(op.red + i);
        T bn[D], t[D], xn[D], ax[D];
#pragma unroll
        for (int k = 0; k < D; ++k) bn[k] = __ldg(op.b + (size_t)k * ld + n);
        nsum(op, n, op.x, t);
#pragma unroll
        for (int k = 0; k < D; ++k) t[k] = bn[k] + op.sc[k] * t[k];
        precond_apply<D, T>(op, n, t, xn);
        block_apply<D, T>(op, n, xn, op.x, ax);
        T rr2 = T(0), b2 = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          rr2 += (bn[k] - ax[k]) * (bn[k] - ax[k]);
          b2 += bn[k] * bn[k];
          op.x[(size_t)k * ld + n] = xn[k];
        }
        krr.add(rr2);
        kbb.add(b2);
      }
    }
    if (!grid_sync(a.bar, &sh_flag)) return false;
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int r = unit_rhs(u), c = unit_chunk(u);
      if (!sel(r)) continue;
      const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
      T *R = Rv + (size_t)r * a.vs, *Uu = UUv + (size_t)r * a.vs;
      T *P = PPv + (size_t)r * a.vs, *Sv = SSv + (size_t)r * a.vs;
      int i0, i1;
      list_chunk(op, op.n_black, c, i0, i1);
      for (int i = i0 + U.lane; i < i1; i += 32) {
        const int n = __ldg(op.black + i);
        T xn[D], bn[D], ax[D], rn[D], un[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          xn[k] = op.x[(size_t)k * ld + n];
          bn[k] = __ldg(op.b + (size_t)k * ld + n);
        }
        block_apply<D, T>(op, n, xn, op.x, ax);
#pragma unroll
        for (int k = 0; k < D; ++k) rn[k] = bn[k] - ax[k];
        precond_apply<D, T>(op, n, rn, un);
        T g = T(0), rr2 = T(0), b2 = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const size_t o = (size_t)k * ld + n;
          R[o] = rn[k];
          Uu[o] = un[k];
          P[o] = T(0);
          Sv[o] = T(0);
          g += rn[k] * un[k];
          rr2 += rn[k] * rn[k];
          b2 += bn[k] * bn[k];
        }
        kg.add(g);
        krr.add(rr2);
        kbb.add(b2);
      }
    }
    if (!grid_sync(a.bar, &sh_flag)) return false;
    rb_red_phase(sel);
    if (!grid_sync(a.bar, &sh_flag)) return false;
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int r = unit_rhs(u), c = unit_chunk(u);
      if (!sel(r)) continue;
      const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
      const T* Uu = UUv + (size_t)r * a.vs;
      T* Wv = WWv + (size_t)r * a.vs;
      int i0, i1;
      list_chunk(op, op.n_black, c, i0, i1);
      for (int i = i0 + U.lane; i < i1; i += 32) {
        const int n = __ldg(op.black + i);
        T un[D], wn[D];
#pragma unroll
        for (int k = 0; k < D; ++k) un[k] = Uu[(size_t)k * ld + n];
        block_apply<D, T>(op, n, un, Uu, wn);
        T dl = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          dl += wn[k] * un[k];
          Wv[(size_t)k * ld + n] = wn[k];
        }
        kd.add(dl);
      }
    }
    if (U.gw < U.units) {
      double acc[4] = {kg.value(), kd.value(), krr.value(), kbb.value()};
      write_partials(U.gw, acc, 0xFu);
    }
    return true;
  };
  // one iteration for the active right-hand sides: black local update (r'u, r'r), red phase,
  // black product (w'u); the caller reduces
  auto iterate_rb = [&]() -> bool {
    KSum<T> kg, kr, kd;
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int r = unit_rhs(u), c = unit_chunk(u);
      if (__ldcg(&a.st[r].active) != 1) continue;
      const T al = (T)__ldcg(&a.st[r].alpha), be = (T)__ldcg(&a.st[r].beta);
      const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
      T *x = op.x, *R = Rv + (size_t)r * a.vs, *Uu = UUv + (size_t)r * a.vs;
      T *P = PPv + (size_t)r * a.vs, *Sv = SSv + (size_t)r * a.vs;
      const T* Wv = WWv + (size_t)r * a.vs;
      int i0, i1;
      list_chunk(op, op.n_black, c, i0, i1);
      for (int i = i0 + U.lane; i < i1; i += 32) {
        const int n = __ldg(op.black + i);
        T rn[D], un[D], pk[D], sk[D], xk[D], wk[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const size_t o = (size_t)k * ld + n;
          un[k] = Uu[o];
          pk[k] = P[o];
          wk[k] = Wv[o];
          sk[k] = Sv[o];
          xk[k] = x[o];
          rn[k] = R[o];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          pk[k] = un[k] + be * pk[k];
          sk[k] = wk[k] + be * sk[k];
          xk[k] += al * pk[k];
          rn[k] -= al * sk[k];
        }
        precond_apply<D, T>(op, n, rn, un);
        T g = T(0), rr2 = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const size_t o = (size_t)k * ld + n;
          P[o] = pk[k];
          Sv[o] = sk[k];
          x[o] = xk[k];
          R[o] = rn[k];
          Uu[o] = un[k];
          g += rn[k] * un[k];
          rr2 += rn[k] * rn[k];
        }
        kg.add(g);
        kr.add(rr2);
      }
    }
    if (!grid_sync(a.bar, &sh_flag)) return false;
    rb_red_phase([&](int r) { return __ldcg(&a.st[r].active) == 1; });
    if (!grid_sync(a.bar, &sh_flag)) return false;
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int r = unit_rhs(u), c = unit_chunk(u);
      if (__ldcg(&a.st[r].active) != 1) continue;
      const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
      const T* Uu = UUv + (size_t)r * a.vs;
      T* Wv = WWv + (size_t)r * a.vs;
      int i0, i1;
      list_chunk(op, op.n_black, c, i0, i1);
      for (int i = i0 + U.lane; i < i1; i += 32) {
        const int n = __ldg(op.black + i);
        T un[D], wn[D];
#pragma unroll
        for (int k = 0; k < D; ++k) un[k] = Uu[(size_t)k * ld + n];
        block_apply<D, T>(op, n, un, Uu, wn);
        T dl = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          dl += wn[k] * un[k];
          Wv[(size_t)k * ld + n] = wn[k];
        }
        kd.add(dl);
      }
    }
    if (U.gw < U.units) {
      double acc[4] = {kg.value(), kd.value(), kr.value(), 0.0};
      write_partials(U.gw, acc, 0x7u);
    }
    return true;
  };
  auto restart_pass = [&](bool first) -> bool {
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int r = unit_rhs(u), c = unit_chunk(u);
      const int act = first ? 1 : __ldcg(&a.st[r].active);
      if (!first && act != 2) continue;
      const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
      const T* b = op.b;
      T *x = op.x, *R = Rv + (size_t)r * a.vs, *Uu = UUv + (size_t)r * a.vs;
      T *P = PPv + (size_t)r * a.vs, *Sv = SSv + (size_t)r * a.vs;
      const int n1 = min(op.N, (c + 1) * op.cs);
      for (int n = c * op.cs + U.lane; n < n1; n += 32) {
        T xn[D], ax[D], rn[D], un[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xn[k] = x[(size_t)k * ld + n];
        block_apply<D, T>(op, n, xn, x, ax);
#pragma unroll
        for (int k = 0; k < D; ++k) rn[k] = __ldg(b + (size_t)k * ld + n) - ax[k];
        precond_apply<D, T>(op, n, rn, un);
        if (a.ssor) {
#pragma unroll
          for (int k = 0; k < D; ++k) un[k] *= (T)a.omega;   // SSOR phase 1
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          R[(size_t)k * ld + n] = rn[k];
          Uu[(size_t)k * ld + n] = un[k];
          P[(size_t)k * ld + n] = T(0);
          Sv[(size_t)k * ld + n] = T(0);
        }
      }
    }
    if (a.ssor && !ssor_phases([&](int r) { return first || __ldcg(&a.st[r].active) == 2; }))
      return false;
    if (!grid_sync(a.bar, &sh_flag)) return false;
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int r = unit_rhs(u), c = unit_chunk(u);
      const int act = first ? 1 : __ldcg(&a.st[r].active);
      KSum<T> ks[4];
      if (first || act == 2) {
        const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
        const T* b = op.b;
        const T* R = Rv + (size_t)r * a.vs;
        const T* Uu = UUv + (size_t)r * a.vs;
        T* Wv = WWv + (size_t)r * a.vs;
        const int n1 = min(op.N, (c + 1) * op.cs);
        for (int n = c * op.cs + U.lane; n < n1; n += 32) {
          T un[D], wn[D], rk[D], bk[D];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            un[k] = Uu[(size_t)k * ld + n];
            rk[k] = R[(size_t)k * ld + n];
            bk[k] = __ldg(b + (size_t)k * ld + n);
          }
          block_apply<D, T>(op, n, un, Uu, wn);
          T g = T(0), dl = T(0), rr2 = T(0), b2 = T(0);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            g += rk[k] * un[k];
            dl += wn[k] * un[k];
            rr2 += rk[k] * rk[k];
            b2 += bk[k] * bk[k];
          }
#pragma unroll
          for (int k = 0; k < D; ++k) Wv[(size_t)k * ld + n] = wn[k];
          ks[0].add(g);
          ks[1].add(dl);
          ks[2].add(rr2);
          ks[3].add(b2);
        }
      }
      double acc[4] = {ks[0].value(), ks[1].value(), ks[2].value(), ks[3].value()};
      write_partials(u, acc, 0xFu);
    }
    return true;
  };

  int any_active = 0, any_pending = 0;
  // the reduced-system path exists for FP64 solves only (the FP32 storage serves the probes,
  // which keep block-Jacobi); a.reduced is ignored in FP32
  constexpr bool kRB = sizeof(T) == 8;
  const bool rb = kRB && a.reduced;
  if constexpr (kRB) {
    if (!(rb ? restart_pass_rb(true) : restart_pass(true))) return;
  } else {
    if (!restart_pass(true)) return;
  }
  if (!mrhs_reduce(a, U, 0, true, sh_int, &any_active, &any_pending)) return;
  while (any_active || any_pending) {
    bool handled = false;
    if constexpr (kRB) {
      if (any_active && rb) {
        if (!iterate_rb()) return;
        if (!mrhs_reduce(a, U, 1, false, sh_int, &any_active, &any_pending)) return;
        handled = true;
      }
    }
    if (handled) {
    } else if (any_active) {
      // local update of active right-hand sides, with the partials r'u and r'r of the
      // updated vectors (columns 0 and 2 of the unit's row)
      for (int u = U.gw; u < U.units; u += U.nw) {
        const int r = unit_rhs(u), c = unit_chunk(u);
        if (__ldcg(&a.st[r].active) != 1) continue;
        KSum<T> kg, kr;
        const T al = (T)__ldcg(&a.st[r].alpha), be = (T)__ldcg(&a.st[r].beta);
        const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
        T *x = op.x, *R = Rv + (size_t)r * a.vs, *Uu = UUv + (size_t)r * a.vs;
        T *P = PPv + (size_t)r * a.vs, *Sv = SSv + (size_t)r * a.vs;
        const T* Wv = WWv + (size_t)r * a.vs;
        const int n0 = c * op.cs;
        const int n1 = min(op.N, (c + 1) * op.cs);
        auto update = [&](int n, T* un, T* pk, T* wk, T* sk, T* xk, T* rn) {
#pragma unroll
          for (int k = 0; k < D; ++k) {
            pk[k] = un[k] + be * pk[k];
            sk[k] = wk[k] + be * sk[k];
            xk[k] += al * pk[k];
            rn[k] -= al * sk[k];
          }
          precond_apply<D, T>(op, n, rn, un);
          if (a.ssor) {
#pragma unroll
            for (int q = 0; q < D; ++q) un[q] *= (T)a.omega;   // SSOR phase 1
          }
          T g = T(0), rr2 = T(0);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const size_t o = (size_t)k * ld + n;
            P[o] = pk[k];
            Sv[o] = sk[k];
            x[o] = xk[k];
            R[o] = rn[k];
            Uu[o] = un[k];
            g += rn[k] * un[k];
            rr2 += rn[k] * rn[k];
          }
          kg.add(g);
          kr.add(rr2);
        };
        if constexpr (kStaged<T>) {
          // The six vectors of the next group of 32 voxels stream into this warp's shared
          // stage (cp.async) while the current group is updated: every lane reads back only
          // the column it copied itself, so no warp synchronisation is needed.
          T* st0 = stage + (size_t)(threadIdx.x >> 5) * 2 * (6 * D) * 32;
          const T* src[6] = {Uu, P, Wv, Sv, x, R};
          auto issue = [&](T* buf, int g0) {
            const int n = g0 + U.lane;
            const bool ok = n < n1;
            const int nn = ok ? n : n0;
#pragma unroll
            for (int v = 0; v < 6; ++v)
#pragma unroll
              for (int k = 0; k < D; ++k)
                cp_async<sizeof(T)>(buf + (size_t)(v * D + k) * 32 + U.lane, src[v] + (size_t)k * ld + nn, ok);
            cp_async_commit();
          };
          if (n0 < n1) issue(st0, n0);
          for (int g0 = n0; g0 < n1; g0 += 32) {
            T* cur = st0 + (size_t)(((g0 - n0) >> 5) & 1) * (6 * D) * 32;
            T* nxt = st0 + (size_t)((((g0 - n0) >> 5) + 1) & 1) * (6 * D) * 32;
            if (g0 + 32 < n1) issue(nxt, g0 + 32);
            else cp_async_commit();               // empty group keeps the wait count uniform
            cp_async_wait<1>();
            const int n = g0 + U.lane;
            if (n < n1) {
              T un[D], pk[D], wk[D], sk[D], xk[D], rn[D];
#pragma unroll
              for (int k = 0; k < D; ++k) {
                un[k] = cur[(0 * D + k) * 32 + U.lane];
                pk[k] = cur[(1 * D + k) * 32 + U.lane];
                wk[k] = cur[(2 * D + k) * 32 + U.lane];
                sk[k] = cur[(3 * D + k) * 32 + U.lane];
                xk[k] = cur[(4 * D + k) * 32 + U.lane];
                rn[k] = cur[(5 * D + k) * 32 + U.lane];
              }
              update(n, un, pk, wk, sk, xk, rn);
            }
          }
          cp_async_wait<0>();
        } else {
          for (int n = n0 + U.lane; n < n1; n += 32) {
            // all loads first: the six vectors are distinct arrays, but the compiler cannot
            // prove it, and interleaved stores would serialise the loads
            T rn[D], un[D], pk[D], sk[D], xk[D], wk[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
              const size_t o = (size_t)k * ld + n;
              un[k] = Uu[o];
              pk[k] = P[o];
              wk[k] = Wv[o];
              sk[k] = Sv[o];
              xk[k] = x[o];
              rn[k] = R[o];
            }
            update(n, un, pk, wk, sk, xk, rn);
          }
        }
        double acc[4] = {kg.value(), 0.0, kr.value(), 0.0};
        write_partials(u, acc, a.ssor ? 0x4u : 0x5u);   // with SSOR, r'u follows the phases
      }
      if (a.ssor && !ssor_phases([&](int r) { return __ldcg(&a.st[r].active) == 1; })) return;
      if (!grid_sync(a.bar, &sh_flag)) return;
      // w = B~ u and the partial w'u (column 1)
      for (int u = U.gw; u < U.units; u += U.nw) {
        const int r = unit_rhs(u), c = unit_chunk(u);
        if (__ldcg(&a.st[r].active) != 1) continue;
        KSum<T> kd, kg;
        const RhsOp<D, T> op = rhs_op<D, T>(a, U, r);
        const size_t ld = op.ld;
        const T* Uu = UUv + (size_t)r * a.vs;
        const T* R = Rv + (size_t)r * a.vs;
        T* Wv = WWv + (size_t)r * a.vs;
        const int n1 = min(op.N, (c + 1) * op.cs);
        for (int n = c * op.cs + U.lane; n < n1; n += 32) {
          T un[D], wn[D];
#pragma unroll
          for (int k = 0; k < D; ++k) un[k] = Uu[(size_t)k * ld + n];
          block_apply<D, T>(op, n, un, Uu, wn);
          T dl = T(0), g = T(0);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            dl += wn[k] * un[k];
            Wv[(size_t)k * ld + n] = wn[k];
          }
          if (a.ssor) {
#pragma unroll
            for (int k = 0; k < D; ++k) g += R[(size_t)k * ld + n] * un[k];
            kg.add(g);
          }
          kd.add(dl);
        }
        double acc[4] = {kg.value(), kd.value(), 0.0, 0.0};
        write_partials(u, acc, a.ssor ? 0x3u : 0x2u);
      }
      if (!mrhs_reduce(a, U, 1, false, sh_int, &any_active, &any_pending)) return;
    } else {
      // every moving RHS has stopped: confirm the pending ones with the true residual
      bool ok = true;
      if constexpr (kRB) ok = rb ? restart_pass_rb(false) : restart_pass(false);
      else ok = restart_pass(false);
      if (!ok) return;
      if (!mrhs_reduce(a, U, 0, false, sh_int, &any_active, &any_pending)) return;
    }
  }
  // states are final (the last reduction's barrier has been passed): accumulate the tally
  if (a.tally != nullptr && blockIdx.x == 0) {
    for (int r = threadIdx.x; r < a.S; r += blockDim.x) {
      const RhsState st = load_state(a.st + r);
      MrhsTally& t = a.tally[r];
      t.iters += st.total;
      t.solves += 1;
      if (st.status != 0 && t.status_any == 0) t.status_any = st.status;
      t.rel_res = st.bb > 0.0 ? sqrt(st.rr / st.bb) : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Right-hand-side tiles (FP32 storage, one shared matrix, block-Jacobi or no preconditioner:
// the probe solves). The S right-hand sides are stored in groups of R interleaved per voxel
// and component, element (i, k, n) at [(i / R) D ld R + (k ld + n) R + i % R], so that one
// thread updates R right-hand sides of one voxel with R-wide loads and stores, and every
// block, factor and neighbour-index load serves R right-hand sides. Units are (group of R,
// voxel chunk); each unit writes the partial row (chunk * S + r) of each of its right-hand
// sides r, so the reducing barrier and the scalar logic are those of k_mrhs.
// ---------------------------------------------------------------------------------------
template <int R>
struct TileVec;
template <>
struct TileVec<2> {
  __device__ __forceinline__ static void ld(const float* p, float* v) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  }
  __device__ __forceinline__ static void st(float* p, const float* v) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
};
template <>
struct TileVec<4> {
  __device__ __forceinline__ static void ld(const float* p, float* v) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
  __device__ __forceinline__ static void st(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

// Two CTAs per SM for tiles of 2 (128 registers); one for tiles of 4, whose R-wide
// vectors of D components need the whole register file of the CTA.
template <int D, int R>
__global__ void __launch_bounds__(MRHS_THREADS, R >= 4 ? 1 : 2) k_mrhs_tile(MrhsArgs a) {
  __shared__ int sh_int[4];
  __shared__ int sh_flag;
  using V = TileVec<R>;
  const size_t ld = a.ld;
  const int S = a.S, G = S / R;
  Units U;   // (first stays null: every right-hand side has U.chunks units)
  U.S = S;
  U.nw = (gridDim.x * blockDim.x) >> 5;
  U.gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  U.lane = threadIdx.x & 31;
  U.chunks = U.nw / G > 0 ? U.nw / G : 1;
  U.units = G * U.chunks;
  {
    const int cs = (a.N + U.chunks - 1) / U.chunks;
    U.csize = ((cs + 31) / 32) * 32;
  }
  grid_barrier_start(a.bar);
  const size_t gs = (size_t)D * ld * R;    // floats per group
  const float* B = static_cast<const float*>(a.blocks);
  const float* M = static_cast<const float*>(a.mfac);
  float sc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) sc[k] = (float)__ldg(a.scale + k);
  float cw6[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) cw6[d] = (float)a.cw[d >> 1];
  auto at = [&](void* base, int g, int k, int n) {
    return static_cast<float*>(base) + (size_t)g * gs + ((size_t)k * ld + n) * R;
  };
  auto cat = [&](const void* base, int g, int k, int n) {
    return static_cast<const float*>(base) + (size_t)g * gs + ((size_t)k * ld + n) * R;
  };
  // y = B~ v for the R right-hand sides of group g at voxel n (v: this voxel's values)
  auto apply = [&](int g, int n, float (*v)[R], const void* Vb, float (*y)[R]) {
    int nb[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = d < a.ndir ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float acc[R];
#pragma unroll
      for (int q = 0; q < R; ++q) acc[q] = 0.f;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float bij = __ldg(B + (size_t)(i >= j ? tri(i, j) : tri(j, i)) * ld + n);
#pragma unroll
        for (int q = 0; q < R; ++q) acc[q] += bij * v[j][q];
      }
#pragma unroll
      for (int q = 0; q < R; ++q) y[i][q] = acc[q];
    }
    // + scale .* sum_d c_d (v - v_m) over the in-mask neighbours
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (nb[d] >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float vm[R];
          V::ld(cat(Vb, g, k, nb[d]), vm);
#pragma unroll
          for (int q = 0; q < R; ++q) y[k][q] += sc[k] * cw6[d] * (v[k][q] - vm[q]);
        }
      }
    }
  };
  auto precond = [&](int n, float (*r)[R], float (*z)[R]) {
    if (M == nullptr) {
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int q = 0; q < R; ++q) z[k][q] = r[k][q];
      return;
    }
    float L[ntri(D)];
#pragma unroll
    for (int e = 0; e < ntri(D); ++e) L[e] = __ldg(M + (size_t)e * ld + n);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      float rq[D], zq[D];
#pragma unroll
      for (int k = 0; k < D; ++k) rq[k] = r[k][q];
      chol_solve_invdiag<D>(L, rq, zq);
#pragma unroll
      for (int k = 0; k < D; ++k) z[k][q] = zq[k];
    }
  };
  auto write_rows = [&](int g, int c, KSum<float> (*acc)[4], unsigned cols) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      double v4[4] = {acc[q][0].value(), acc[q][1].value(), acc[q][2].value(), acc[q][3].value()};
      const double v = warp_reduce4(v4);
      const int u = c * S + g * R + q;
      if ((U.lane & 7) == 0 && ((cols >> (U.lane >> 3)) & 1u)) a.part[(size_t)u * 4 + (U.lane >> 3)] = v;
    }
  };
  auto state_of = [&](int r) { return __ldcg(&a.st[r].active); };
  // (re)start: r = b - B~ x, u = M^-1 r, p = s = 0 for the selected right-hand sides, then
  // w = B~ u and the partials (r'u, w'u, r'r, b'b)
  auto restart = [&](bool first) -> bool {
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int g = u % G, c = u / G;
      bool sel[R], any = false;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        sel[q] = first || state_of(g * R + q) == 2;
        any |= sel[q];
      }
      if (!any) continue;
      const int n1 = min(a.N, (c + 1) * U.csize);
      for (int n = c * U.csize + U.lane; n < n1; n += 32) {
        float xn[D][R], ax[D][R], rn[D][R], zn[D][R], bn[D][R], zero[R];
#pragma unroll
        for (int q = 0; q < R; ++q) zero[q] = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          V::ld(cat(a.x, g, k, n), xn[k]);
          V::ld(cat(a.b, g, k, n), bn[k]);
        }
        apply(g, n, xn, a.x, ax);
#pragma unroll
        for (int k = 0; k < D; ++k)
#pragma unroll
          for (int q = 0; q < R; ++q) rn[k][q] = bn[k][q] - ax[k][q];
        precond(n, rn, zn);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float ro[R], uo[R], po[R], so[R];
          if (!first) {
            V::ld(cat(a.r, g, k, n), ro);
            V::ld(cat(a.u, g, k, n), uo);
            V::ld(cat(a.p, g, k, n), po);
            V::ld(cat(a.s, g, k, n), so);
          }
#pragma unroll
          for (int q = 0; q < R; ++q) {
            ro[q] = sel[q] ? rn[k][q] : ro[q];
            uo[q] = sel[q] ? zn[k][q] : uo[q];
            po[q] = sel[q] ? 0.f : po[q];
            so[q] = sel[q] ? 0.f : so[q];
          }
          V::st(at(a.r, g, k, n), ro);
          V::st(at(a.u, g, k, n), uo);
          V::st(at(a.p, g, k, n), po);
          V::st(at(a.s, g, k, n), so);
        }
        (void)zero;
      }
    }
    if (!grid_sync(a.bar, &sh_flag)) return false;
    for (int u = U.gw; u < U.units; u += U.nw) {
      const int g = u % G, c = u / G;
      bool sel[R], any = false;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        sel[q] = first || state_of(g * R + q) == 2;
        any |= sel[q];
      }
      KSum<float> acc[R][4];
      if (any) {
        const int n1 = min(a.N, (c + 1) * U.csize);
        for (int n = c * U.csize + U.lane; n < n1; n += 32) {
          float un[D][R], wn[D][R], rn[D][R], bn[D][R];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            V::ld(cat(a.u, g, k, n), un[k]);
            V::ld(cat(a.r, g, k, n), rn[k]);
            V::ld(cat(a.b, g, k, n), bn[k]);
          }
          apply(g, n, un, a.u, wn);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float wo[R];
            if (!first) V::ld(cat(a.w, g, k, n), wo);
#pragma unroll
            for (int q = 0; q < R; ++q) wo[q] = sel[q] ? wn[k][q] : wo[q];
            V::st(at(a.w, g, k, n), wo);
          }
#pragma unroll
          for (int q = 0; q < R; ++q) {
            if (!sel[q]) continue;
            float gg = 0.f, dl = 0.f, rr2 = 0.f, b2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              gg += rn[k][q] * un[k][q];
              dl += wn[k][q] * un[k][q];
              rr2 += rn[k][q] * rn[k][q];
              b2 += bn[k][q] * bn[k][q];
            }
            acc[q][0].add(gg);
            acc[q][1].add(dl);
            acc[q][2].add(rr2);
            acc[q][3].add(b2);
          }
        }
      }
      write_rows(g, c, acc, 0xFu);
    }
    return true;
  };

  int any_active = 0, any_pending = 0;
  if (!restart(true)) return;
  if (!mrhs_reduce(a, U, 0, true, sh_int, &any_active, &any_pending)) return;
  while (any_active || any_pending) {
    if (any_active) {
      // local update (p, s, x, r, u) of the active right-hand sides; partials r'u and r'r
      for (int u = U.gw; u < U.units; u += U.nw) {
        const int g = u % G, c = u / G;
        bool act[R], any = false;
        float al[R], be[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          act[q] = state_of(g * R + q) == 1;
          any |= act[q];
          al[q] = act[q] ? (float)__ldcg(&a.st[g * R + q].alpha) : 0.f;
          be[q] = act[q] ? (float)__ldcg(&a.st[g * R + q].beta) : 0.f;
        }
        KSum<float> acc[R][4];
        if (any) {
          const int n1 = min(a.N, (c + 1) * U.csize);
          for (int n = c * U.csize + U.lane; n < n1; n += 32) {
            float rn[D][R], zn[D][R];
#pragma unroll
            for (int k = 0; k < D; ++k) {
              float uk[R], pk[R], wk[R], sk[R], xk[R];
              V::ld(cat(a.u, g, k, n), uk);
              V::ld(cat(a.p, g, k, n), pk);
              V::ld(cat(a.w, g, k, n), wk);
              V::ld(cat(a.s, g, k, n), sk);
              V::ld(cat(a.x, g, k, n), xk);
              V::ld(cat(a.r, g, k, n), rn[k]);
#pragma unroll
              for (int q = 0; q < R; ++q) {
                if (act[q]) {
                  pk[q] = uk[q] + be[q] * pk[q];
                  sk[q] = wk[q] + be[q] * sk[q];
                  xk[q] += al[q] * pk[q];
                  rn[k][q] -= al[q] * sk[q];
                }
              }
              V::st(at(a.p, g, k, n), pk);
              V::st(at(a.s, g, k, n), sk);
              V::st(at(a.x, g, k, n), xk);
            }
            // z = M^-1 r; for a right-hand side that does not move, r is unchanged and the
            // same arithmetic reproduces its u exactly
            precond(n, rn, zn);
#pragma unroll
            for (int k = 0; k < D; ++k) {
              V::st(at(a.r, g, k, n), rn[k]);
              V::st(at(a.u, g, k, n), zn[k]);
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
              if (!act[q]) continue;
              float gg = 0.f, rr2 = 0.f;
#pragma unroll
              for (int k = 0; k < D; ++k) {
                gg += rn[k][q] * zn[k][q];
                rr2 += rn[k][q] * rn[k][q];
              }
              acc[q][0].add(gg);
              acc[q][2].add(rr2);
            }
          }
        }
        write_rows(g, c, acc, 0x5u);
      }
      if (!grid_sync(a.bar, &sh_flag)) return;
      // w = B~ u and w'u (column 1)
      for (int u = U.gw; u < U.units; u += U.nw) {
        const int g = u % G, c = u / G;
        bool act[R], any = false;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          act[q] = state_of(g * R + q) == 1;
          any |= act[q];
        }
        KSum<float> acc[R][4];
        if (any) {
          const int n1 = min(a.N, (c + 1) * U.csize);
          for (int n = c * U.csize + U.lane; n < n1; n += 32) {
            float un[D][R], wn[D][R];
#pragma unroll
            for (int k = 0; k < D; ++k) V::ld(cat(a.u, g, k, n), un[k]);
            apply(g, n, un, a.u, wn);
            float wo[D][R];
            bool all = true;
#pragma unroll
            for (int q = 0; q < R; ++q) all &= act[q];
            if (!all) {
#pragma unroll
              for (int k = 0; k < D; ++k) V::ld(cat(a.w, g, k, n), wo[k]);
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
#pragma unroll
              for (int q = 0; q < R; ++q) wo[k][q] = act[q] ? wn[k][q] : wo[k][q];
              V::st(at(a.w, g, k, n), wo[k]);
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
              if (!act[q]) continue;
              float dl = 0.f;
#pragma unroll
              for (int k = 0; k < D; ++k) dl += wn[k][q] * un[k][q];
              acc[q][1].add(dl);
            }
          }
        }
        write_rows(g, c, acc, 0x2u);
      }
      if (!mrhs_reduce(a, U, 1, false, sh_int, &any_active, &any_pending)) return;
    } else {
      if (!restart(false)) return;
      if (!mrhs_reduce(a, U, 0, false, sh_int, &any_active, &any_pending)) return;
    }
  }
}

template <int D, int R>
static cudaError_t launch_tile(const MrhsArgs& a, int nsm, cudaStream_t stream, int* units_out) {
  const void* kern = (const void*)k_mrhs_tile<D, R>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, MRHS_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int G = a.S / R;
  const long long want_warps = (long long)G * ((a.N + 31) / 32);
  long long grid = (want_warps * 32 + MRHS_THREADS - 1) / MRHS_THREADS;
  if (grid > (long long)nsm * per_sm) grid = (long long)nsm * per_sm;
  if (grid < 1) grid = 1;
  const int nw = (int)grid * (MRHS_THREADS / 32);
  const int chunks = nw / G > 0 ? nw / G : 1;
  if (units_out) *units_out = G * chunks;
  e = reset_grid_barrier(a.bar, stream);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel(kern, dim3((unsigned)grid), dim3(MRHS_THREADS), args, 0, stream);
}

namespace mrhs_detail {

template <int D>
cudaError_t launch_d(const MrhsArgs& a, cudaStream_t stream, int* units_out) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (a.sm_cap > 0 && a.sm_cap < nsm) nsm = a.sm_cap;
  if (a.tile > 1) {
    if (!a.f32 || a.ssor || a.reduced || a.tab != nullptr || a.uneven || a.S % a.tile != 0)
      return cudaErrorInvalidValue;
    if (a.tile == 2) return launch_tile<D, 2>(a, nsm, stream, units_out);
    if (a.tile == 4) return launch_tile<D, 4>(a, nsm, stream, units_out);
    return cudaErrorInvalidValue;
  }
  if (a.uneven && (a.tab == nullptr || a.S > MRHS_UNEVEN_MAX_S)) return cudaErrorInvalidValue;
  const void* kern = a.f32 ? (const void*)k_mrhs<D, float> : (const void*)k_mrhs<D, double>;
  const size_t shm = a.f32 ? mrhs_stage_bytes<D, float>() : mrhs_stage_bytes<D, double>();
  if (shm > 0) {
    cudaError_t ea = raise_smem_limit(kern, shm);
    if (ea != cudaSuccess) return ea;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, MRHS_THREADS, shm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // enough warps for every RHS and for a chunk of at least 32 voxels per warp
  const long long want_warps = (long long)a.S * ((a.N + 31) / 32);
  long long grid = (want_warps * 32 + MRHS_THREADS - 1) / MRHS_THREADS;
  if (grid > (long long)nsm * per_sm) grid = (long long)nsm * per_sm;
  if (grid < 1) grid = 1;
  const int nw = (int)grid * (MRHS_THREADS / 32);
  int chunks = nw / a.S;
  if (chunks < 1) chunks = 1;
  if (units_out) *units_out = a.S * chunks;
  // the reduced-system path keeps one unit per warp: with more right-hand sides than warps it
  // runs the equivalent SSOR form (omega = 1) instead
  MrhsArgs b = a;
  if (b.reduced && b.S > nw) {
    b.reduced = 0;
    b.ssor = 1;
    b.omega = 1.0;
  }
  e = reset_grid_barrier(b.bar, stream);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&b};
  return cudaLaunchCooperativeKernel(kern, dim3((unsigned)grid), dim3(MRHS_THREADS), args, shm, stream);
}

template <int D>
int max_units_d(int S) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mrhs<D, double>, MRHS_THREADS, 0);
  const int nw = nsm * (per_sm > 0 ? per_sm : 1) * (MRHS_THREADS / 32);
  const int chunks = nw / S > 0 ? nw / S : 1;
  return S * chunks;
}

}  // namespace mrhs_detail

// explicit instantiation of the launchers for one D (kernels_mrhs_d*.cu)
#define BFMRI_MRHS_INSTANTIATE(d)                                                         \
  template cudaError_t mrhs_detail::launch_d<d>(const MrhsArgs&, cudaStream_t, int*);    \
  template int mrhs_detail::max_units_d<d>(int);

}  // namespace bfmri
