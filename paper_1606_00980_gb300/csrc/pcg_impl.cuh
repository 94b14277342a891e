// Persistent, cooperative preconditioned conjugate gradients for the W and A draws
// (Algorithm 2, step 7: solve B~ w = b approximately by PCG from a starting value, until the
// relative residual ||B~ w - b|| / ||b|| is below delta; Section 3.1).
//
// One launch runs the whole solve. The recurrence is the Chronopoulos & Gear (1989) form of
// preconditioned CG, in which the two inner products of an iteration are formed together:
//   p = u + beta p,  s = w + beta s,  x += a p,  r -= a s,  u = M^-1 r      (local)
//   --- grid barrier (neighbour values of u are complete) ---
//   w = B~ u,  gamma = r'u,  delta = w'u,  rr = r'r                         (stencil + block)
//   --- reducing grid barrier ---
//   beta = gamma / gamma_old,  a = gamma / (delta - beta gamma / a_old)
// so each iteration has one matrix product, one preconditioner application, one plain and
// one reducing barrier. When the recursive residual reaches the tolerance, the true residual
// b - B~ x is formed in FP64 and confirms the stop (or restarts the recurrence from it).
//
// Two variants:
//  * resident: one voxel per thread, one CTA per SM; the per-voxel block and preconditioner
//    factor are staged once in shared memory and all vectors stay in registers, so an
//    iteration only exchanges u through L2;
//  * streaming: any N; vectors live in global memory (structure of arrays).
// All reductions are fixed-order, so a solve is bit-reproducible: FP64 sums (grid_allreduce4)
// for the FP64 solves and the outer residuals of the mixed solves, float-float sums
// (grid_allreduce4_ff) for the FP32 inner iterations of the mixed solves.
#pragma once
// The solver kernels and their launchers, included by the translation units that instantiate
// them for groups of D (kernels_pcg_d*.cu) so that the heaviest compile is spread over
// several parallel jobs; kernels_pcg.cu holds the dispatch by D.
#include <algorithm>

#include "pcg.cuh"

namespace bfmri {

namespace {

constexpr int RES_MAX_THREADS = 384;
// The reduced-system kernel keeps one more vector per voxel (b^): at most 352 threads, so
// that it may take 184 registers a thread (N <= 152 x 352 voxels on one GB300)
constexpr int RB_MAX_THREADS = 352;
constexpr int RES_MAX_D = 8;
// prior variants of the resident kernels (separate instantiations, so that the graph-Laplacian
// kernels keep their register allocation): direction weights, the anisotropic prior's
// per-direction scales (a.scale3), per-edge factors (a.ce, slot weights per voxel in shared
// memory)
constexpr int PRIOR_DIR = 0, PRIOR_SCALE3 = 1, PRIOR_EDGE = 2;
// the L'L prior (block-Jacobi resident kernel): each product publishes t = L v (a.t) and
// reads its neighbours after a grid barrier
constexpr int PRIOR_LTL = 3;

__device__ __forceinline__ double ldx(const double* p) { return __ldcg(p); }

__device__ __forceinline__ float ldx(const float* p) { return __ldcg(p); }

// out = B v + s .* (deg v - sum_m c_m V[m])  (B packed, entry e at Bp[e * bs]; c: the edge
// weight of each neighbour slot, deg their sum over the in-mask neighbours); element type T.
template <int D, typename T>
__device__ __forceinline__ void amul(const T* __restrict__ Bp, int bs, const T* s,
                                     const int* nb, const T* cw6, T degT, const T* v,
                                     const T* V, size_t ld, T* out) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) acc += Bp[(size_t)(i >= j ? tri(i, j) : tri(j, i)) * bs] * v[j];
    out[i] = acc;
  }
  T sum[D];
#pragma unroll
  for (int k = 0; k < D; ++k) sum[k] = T(0);
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    if (nb[d] >= 0) {
#pragma unroll
      for (int k = 0; k < D; ++k) sum[k] += cw6[d] * ldx(V + (size_t)k * ld + nb[d]);
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) out[k] += s[k] * (degT * v[k] - sum[k]);
}

// out = B v + sum over the neighbour slots d of s3[d / 2][k] c_d (v_k - V_k[m_d]): the
// anisotropic prior, one scale per direction and component (FP64 streaming solver).
template <int D>
__device__ __forceinline__ void amul_dir(const double* __restrict__ Bp, int bs, const double (*s3)[DMAX],
                                         const int* nb, const double* cw6, const double* v,
                                         const double* V, size_t ld, double* out) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) acc += Bp[(size_t)(i >= j ? tri(i, j) : tri(j, i)) * bs] * v[j];
    out[i] = acc;
  }
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    if (nb[d] >= 0) {
#pragma unroll
      for (int k = 0; k < D; ++k) out[k] += s3[d >> 1][k] * cw6[d] * (v[k] - ldx(V + (size_t)k * ld + nb[d]));
    }
  }
}

// weighted number of in-mask neighbours (slots past the neighbourhood hold -1)
template <typename T>
__device__ __forceinline__ T degree_of(const int* nb, const T* cw6) {
  T deg = T(0);
#pragma unroll
  for (int d = 0; d < 6; ++d) deg += nb[d] >= 0 ? cw6[d] : T(0);
  return deg;
}

// the edge weight of each neighbour slot (-x, +x, -y, +y, -z, +z) in element type T
template <typename T>
__device__ __forceinline__ void slot_weights(const PcgArgs& a, T* cw6) {
#pragma unroll
  for (int d = 0; d < 6; ++d) cw6[d] = (T)a.cw[d >> 1];
}

// z = (L L')^-1 r with L packed lower (inverted diagonal), entry e at Lp[e * bs].
template <int D, typename T>
__device__ __forceinline__ void minv(const T* __restrict__ Lp, int bs, const T* r, T* z) {
  T y[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T t = r[i];
#pragma unroll
    for (int j = 0; j < i; ++j) t -= Lp[(size_t)tri(i, j) * bs] * y[j];
    y[i] = t * Lp[(size_t)tri(i, i) * bs];
  }
#pragma unroll
  for (int i = D - 1; i >= 0; --i) {
    T t = y[i];
#pragma unroll
    for (int j = i + 1; j < D; ++j) t -= Lp[(size_t)tri(j, i) * bs] * z[j];
    z[i] = t * Lp[(size_t)tri(i, i) * bs];
  }
}

// z = Minv r with Minv symmetric packed (entry e at Mp[e * bs]): D independent row sums,
// no dependent chain as in the two triangular solves.
template <int D, typename T>
__device__ __forceinline__ void symv(const T* __restrict__ Mp, int bs, const T* r, T* z) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j) acc += Mp[(size_t)(i >= j ? tri(i, j) : tri(j, i)) * bs] * r[j];
    z[i] = acc;
  }
}

// Li = L^-1 (packed lower) of a packed Cholesky factor L (lower, inverted diagonal; entry e
// at Mp[e * bs]), column by column by forward substitution.
template <int D, typename T>
__device__ __forceinline__ void lower_inverse(const T* Mp, int bs, T* Li) {
#pragma unroll
  for (int j = 0; j < D; ++j) {
    Li[tri(j, j)] = Mp[(size_t)tri(j, j) * bs];
#pragma unroll
    for (int i = j + 1; i < D; ++i) {
      T acc = T(0);
#pragma unroll
      for (int k = j; k < i; ++k) acc += Mp[(size_t)tri(i, k) * bs] * Li[tri(k, j)];
      Li[tri(i, j)] = -acc * Mp[(size_t)tri(i, i) * bs];
    }
  }
}

// out = L v (lower = true) or L' v (lower = false) for a packed lower-triangular L (entry e
// at Lp[e * bs]): rows of independent sums.
template <int D, typename T, bool lower>
__device__ __forceinline__ void trmv(const T* __restrict__ Lp, int bs, const T* v, T* out) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T acc = T(0);
    if constexpr (lower) {
#pragma unroll
      for (int j = 0; j <= i; ++j) acc += Lp[(size_t)tri(i, j) * bs] * v[j];
    } else {
#pragma unroll
      for (int j = i; j < D; ++j) acc += Lp[(size_t)tri(j, i) * bs] * v[j];
    }
    out[i] = acc;
  }
}

// Replaces a packed Cholesky factor L (lower, inverted diagonal; M = L L') by the packed
// symmetric inverse M^-1 = L^-T L^-1, in place (entry e at Mp[e * bs]).
template <int D, typename T>
__device__ __forceinline__ void factor_to_inverse(T* Mp, int bs) {
  T Li[ntri(D)];   // L^-1, lower, packed
  lower_inverse<D, T>(Mp, bs, Li);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = i; k < D; ++k) acc += Li[tri(k, i)] * Li[tri(k, j)];
      Mp[(size_t)tri(i, j) * bs] = acc;
    }
}

struct Shared {
  double red[32 * 4 + 8];
  double scal[4];   // CG scalars computed once per CTA by thread 0
  int ints[2];
  int flag;
  int code;         // broadcast control code
};

// Reciprocal by Newton-Raphson refinement, x <- x + x (1 - d x), of the hardware's
// approximate FP64 reciprocal: each step squares the relative error, and two steps bring the
// approximation's error to the FP64 rounding level. The CG scalars need no correctly
// rounded quotient, and this is a short dependent chain on the one thread that runs it.
__device__ __forceinline__ double recip_nr(double d) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
  double e = fma(-d, x, 1.0);
  x = fma(x, e, x);
  e = fma(-d, x, 1.0);
  return fma(x, e, x);
}

// 1/gamma and 1/alpha = delta/gamma for a (re)started recurrence with alpha = gamma/delta.
__device__ __forceinline__ void cg_recips(double gam, double del, double& rgam, double& ralpha) {
  rgam = gam > 0.0 ? recip_nr(gam) : 0.0;
  ralpha = del * rgam;
}

// One CG step of the scalar recurrence (Chronopoulos & Gear), evaluated by thread 0 of each
// CTA and broadcast through shared memory. With 1/gamma_old and 1/alpha_old kept from the
// previous step, the critical path holds a single reciprocal (of the new denominator);
// the reciprocals for the next step are formed after the broadcast, while the other threads
// move on. Returns in sh.code: 0 continue, 1 check the true residual, 3 breakdown,
// 7 non-finite.
__device__ __forceinline__ void cg_scalar_step(Shared& sh, double gnew, double dnew, double rr,
                                               double tol2, int it, int max_iter, double& alpha,
                                               double& beta, double& gam, double& rgam,
                                               double& ralpha) {
  if (threadIdx.x == 0) {
    int code = 0;
    double a = alpha, b = beta, g = gam, den = 0.0;
    if (!(isfinite(gnew) && isfinite(dnew) && isfinite(rr))) {
      code = 7;
    } else if (rr <= tol2 || it >= max_iter) {
      code = 1;
    } else {
      b = gnew * rgam;
      den = fma(-(b * gnew), ralpha, dnew);
      if (!(den > 0.0)) {
        code = 3;
      } else {
        a = gnew * recip_nr(den);
        g = gnew;
      }
    }
    sh.scal[0] = a;
    sh.scal[1] = b;
    sh.scal[2] = g;
    sh.scal[3] = den;
    sh.code = code;
  }
  __syncthreads();
  alpha = sh.scal[0];
  beta = sh.scal[1];
  gam = sh.scal[2];
  if (threadIdx.x == 0 && sh.code == 0) {
    rgam = recip_nr(gam);
    ralpha = sh.scal[3] * rgam;
  }
}

// Red-black symmetric SOR: z = M(omega)^-1 r with
//   M(omega) = (Dg + omega L) Dg^-1 (Dg + omega U) / (omega (2 - omega))
// in red-black order (Dg: the voxel blocks B_n + diag(scale) deg_n, whose Cholesky factor is
// mfac; L, U: the couplings -scale_k between neighbours, each joining a red and a black
// voxel). It equals one forward SOR sweep (red, then black voxels) and one backward sweep
// (black, then red) from z = 0. The backward half-sweep of the black voxels only rescales
// them by (2 - omega), so three colour phases remain, with neighbour values exchanged
// between them (u holds z in place):
//   1. every voxel: u_n = omega Dg_n^-1 r_n      (read afterwards only for the red voxels)
//   2. black n:     u_n = (2 - omega) omega Dg_n^-1 (r_n + scale .* sum_m u_m)
//   3. red n:       u_n = (2 - omega) u_n + omega Dg_n^-1 (scale .* sum_m u_m)
// Phase 1 is the solver's block-Jacobi step scaled by omega; phases 2 and 3 are below
// (streaming layout: factor Mf, r and u in global memory; element type T).
template <int D, typename T>
__device__ __forceinline__ void ssor_phase(const PcgArgs& a, const T* s, const T* Mf, const T* R,
                                           T* U, int n, int phase) {
  const size_t ld = a.ld;
  int nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = d < a.ndir ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  T sum[D];
#pragma unroll
  for (int k = 0; k < D; ++k) sum[k] = T(0);
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    if (nb[d] >= 0) {
#pragma unroll
      for (int k = 0; k < D; ++k) sum[k] += (T)a.cw[d >> 1] * ldx(U + (size_t)k * ld + nb[d]);
    }
  }
  T t[D], z[D];
#pragma unroll
  for (int k = 0; k < D; ++k) t[k] = phase == 2 ? R[(size_t)k * ld + n] + s[k] * sum[k] : s[k] * sum[k];
  minv<D, T>(Mf + n, (int)ld, t, z);
  const T omega = (T)a.omega, c = T(2) - omega;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const size_t o = (size_t)k * ld + n;
    U[o] = phase == 2 ? c * omega * z[k] : c * U[o] + omega * z[k];
  }
}

__device__ __forceinline__ void write_ctrl(const PcgArgs& a, int it, int restarts, double rr,
                                          double bb, double rel0, int status) {
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

}  // namespace

// Resident SSOR ownership: the CTA's red voxels take its first threads and its black voxels
// the next ones (stable within each colour), so the warps of each colour phase are uniform.
// In: this thread's voxel n and whether it owns one; out: the colour-sorted voxel, ownership
// and colour.
__device__ __forceinline__ void colour_sort(const PcgArgs& a, int& n, bool& own, bool& is_red) {
  __shared__ int sh_order[RES_MAX_THREADS];
  __shared__ int sh_cnt[2 * (RES_MAX_THREADS / 32)];
  const int t = threadIdx.x, bd = blockDim.x;
  const bool blk = own && a.colour[n] != 0;
  const bool rd = own && !blk;
  const int lane = t & 31, warp = t >> 5, nwc = (bd + 31) >> 5;
  const unsigned mr = __ballot_sync(0xffffffffu, rd), mb = __ballot_sync(0xffffffffu, blk);
  if (lane == 0) {
    sh_cnt[2 * warp] = __popc(mr);
    sh_cnt[2 * warp + 1] = __popc(mb);
  }
  __syncthreads();
  int red_before = 0, black_before = 0, nred = 0, nblack = 0;
  for (int w = 0; w < nwc; ++w) {
    if (w < warp) {
      red_before += sh_cnt[2 * w];
      black_before += sh_cnt[2 * w + 1];
    }
    nred += sh_cnt[2 * w];
    nblack += sh_cnt[2 * w + 1];
  }
  const unsigned below = (1u << lane) - 1u;
  if (rd) sh_order[red_before + __popc(mr & below)] = n;
  if (blk) sh_order[nred + black_before + __popc(mb & below)] = n;
  __syncthreads();
  own = t < nred + nblack;
  n = own ? sh_order[t] : 0;
  is_red = t < nred;
}

// Resident SSOR phases 2 (black voxels) and 3 (red voxels) in element type T (FP64 solves,
// or the FP32 inner iterations of the mixed ones), each after a grid barrier: u and r are this
// thread's registers, Mp its factor in shared memory, U the published u of every voxel.
template <int D, typename T, typename Bar>
__device__ __forceinline__ bool resident_ssor_phases(const PcgArgs& a, Bar& bar, bool own, bool is_red,
                                                     const int* nb, const T* s, const T* Mp, int bd,
                                                     int n, const T* r, T* u, T* U) {
  const T omega = (T)a.omega, c2 = T(2) - omega;
  for (int phase = 2; phase <= 3; ++phase) {
    if (!bar()) return false;
    if (own && (phase == 2) != is_red) {
      T sum[D], tv[D], z[D];
#pragma unroll
      for (int k = 0; k < D; ++k) sum[k] = T(0);
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        if (nb[d] >= 0) {
#pragma unroll
          for (int k = 0; k < D; ++k) sum[k] += (T)a.cw[d >> 1] * ldx(U + (size_t)k * a.ld + nb[d]);
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) tv[k] = phase == 2 ? r[k] + s[k] * sum[k] : s[k] * sum[k];
      minv<D, T>(Mp, bd, tv, z);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        u[k] = phase == 2 ? c2 * omega * z[k] : c2 * u[k] + omega * z[k];
        U[(size_t)k * a.ld + n] = u[k];
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Resident variant.
// ---------------------------------------------------------------------------------------
// PRIOR: PRIOR_SCALE3 (the anisotropic prior's per-direction scales in shared memory) and
// PRIOR_EDGE (per-edge factors: the voxel's six slot weights in shared memory after the
// blocks) run without SSOR.
template <int D, int PRIOR>
__global__ void __launch_bounds__(RES_MAX_THREADS, 1) k_pcg_res(PcgArgs a) {
  constexpr bool ANISO = PRIOR == PRIOR_SCALE3;
  extern __shared__ double smem[];
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  // per-slot edge weights in shared memory (read as broadcasts; no registers held)
  __shared__ double cwd[6];
  __shared__ float cwf[6];
  __shared__ double s3[ANISO ? 3 : 1][ANISO ? DMAX : 1];
  if (threadIdx.x == 0) {
    slot_weights(a, cwd);
    slot_weights(a, cwf);
  }
  if constexpr (ANISO) {
    if (threadIdx.x < 3 * D) s3[threadIdx.x / D][threadIdx.x % D] = a.scale3[threadIdx.x];
  }
  __syncthreads();
  constexpr int NT = ntri(D);
  const int bd = blockDim.x, t = threadIdx.x;
  double* shB = smem;
  double* shM = smem + NT * bd;
  int n = blockIdx.x * a.res_per + t;
  bool own = t < a.res_per && n < a.N;
  bool is_red = true;
  if (a.ssor) colour_sort(a, n, own, is_red);
  const size_t ld = a.ld;
  const bool pre = a.mfac != nullptr;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const int e = tri(i, j);
      shB[e * bd + t] = own ? __ldg(a.blocks + (size_t)e * ld + n) : (i == j ? 1.0 : 0.0);
      shM[e * bd + t] = (own && pre) ? __ldg(a.mfac + (size_t)e * ld + n) : (i == j ? 1.0 : 0.0);
    }
  int nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = (own && d < a.ndir) ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  double* shC = smem + 2 * NT * bd;    // PRIOR_EDGE: slot weights [6][bd]
  if constexpr (PRIOR == PRIOR_EDGE) {
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      double c = cwd[d];
      // the edge's factor is stored at its lower voxel: n for +d, the neighbour for -d
      if (nb[d] >= 0)
        c *= (double)__uint_as_float((unsigned)__ldg(a.ce + (size_t)(d >> 1) * ld + ((d & 1) ? n : nb[d])) << 16);
      shC[d * bd + t] = c;
    }
  }
  auto edge_weights = [&](double* c6) {
#pragma unroll
    for (int d = 0; d < 6; ++d) c6[d] = shC[d * bd + t];
  };
  double degd;
  if constexpr (PRIOR == PRIOR_EDGE) {
    double c6[6];
    edge_weights(c6);
    degd = degree_of<double>(nb, c6);
  } else {
    degd = degree_of<double>(nb, cwd);
  }
  double s[D], x[D], r[D], u[D], w[D], p[D], q[D], bv[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    s[k] = ANISO ? 0.0 : __ldg(a.scale + k);
    x[k] = own ? a.x[(size_t)k * ld + n] : 0.0;
    bv[k] = own ? __ldg(a.b + (size_t)k * ld + n) : 0.0;
    p[k] = 0.0;
    q[k] = 0.0;
  }
  const double* Bp = shB + t;
  const double* Mp = shM + t;
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  // (B~ v)_n with v_n = vn and the vector V for the neighbours
  // false when a grid barrier gave up (the L'L prior's product waits for the other CTAs' t)
  auto product = [&](const double* vn, const double* V, double* out) -> bool {
    if constexpr (ANISO) {
      amul_dir<D>(Bp, bd, s3, nb, cwd, vn, V, ld, out);
    } else if constexpr (PRIOR == PRIOR_EDGE) {
      double c6[6];
      edge_weights(c6);
      amul<D, double>(Bp, bd, s, nb, c6, degd, vn, V, ld, out);
    } else if constexpr (PRIOR == PRIOR_LTL) {
      // t = L v at this voxel, published for the neighbours; then B v + s .* (L t)
      double tn[D], sum[D];
#pragma unroll
      for (int k = 0; k < D; ++k) sum[k] = 0.0;
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        if (nb[d] >= 0) {
#pragma unroll
          for (int k = 0; k < D; ++k) sum[k] += cwd[d] * ldx(V + (size_t)k * ld + nb[d]);
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) tn[k] = degd * vn[k] - sum[k];
      if (own) {
#pragma unroll
        for (int k = 0; k < D; ++k) a.t[(size_t)k * ld + n] = tn[k];
      }
      if (!bar()) return false;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < D; ++j) acc += Bp[(size_t)(i >= j ? tri(i, j) : tri(j, i)) * bd] * vn[j];
        out[i] = acc;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) sum[k] = 0.0;
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        if (nb[d] >= 0) {
#pragma unroll
          for (int k = 0; k < D; ++k) sum[k] += cwd[d] * ldx(a.t + (size_t)k * ld + nb[d]);
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) out[k] += s[k] * (degd * tn[k] - sum[k]);
    } else {
      amul<D, double>(Bp, bd, s, nb, cwd, degd, vn, V, ld, out);
    }
    return true;
  };
  const double omega = a.omega;
  // SSOR phase 1 is the block-Jacobi step scaled by omega (u published by the caller);
  // phases 2 (black voxels) and 3 (red voxels) follow, each after a barrier
  auto ssor_phases = [&]() -> bool {
    return resident_ssor_phases<D, double>(a, bar, own, is_red, nb, s, Mp, bd, n, r, u, a.u);
  };
  // (r, u, w) from the current x, with partials (r'u, w'u, r'r, b'b)
  auto restart = [&](double* tot) -> bool {
    double ax[D];
    if (!product(x, a.x, ax)) return false;
#pragma unroll
    for (int k = 0; k < D; ++k) r[k] = bv[k] - ax[k];
    // SSOR phase 1 (red voxels only: the black ones are overwritten by phase 2 before
    // anyone reads them); the colour-sorted warps keep this branch uniform
    if (!a.ssor) {
      minv<D, double>(Mp, bd, r, u);
    } else if (is_red) {
      minv<D, double>(Mp, bd, r, u);
#pragma unroll
      for (int k = 0; k < D; ++k) u[k] *= omega;
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) u[k] = 0.0;   // defined for threads without a voxel
    }
    if (own) {
#pragma unroll
      for (int k = 0; k < D; ++k) a.u[(size_t)k * ld + n] = u[k];
    }
    if (a.ssor && !ssor_phases()) return false;
    if (!bar()) return false;
    if (!product(u, a.u, w)) return false;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[0] += r[k] * u[k];
      v[1] += w[k] * u[k];
      v[2] += r[k] * r[k];
      v[3] += bv[k] * bv[k];
    }
    return grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };

  double tot[4];
  if (!restart(tot)) return;   // x is the caller's start value, complete before the launch
  double gam = tot[0], del = tot[1], rr = tot[2];
  const double bb = tot[3];
  const double tol2 = a.delta * a.delta * bb;
  const double rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  int it = 0, restarts = 0, status = 0;
  if (!(isfinite(gam) && isfinite(del) && isfinite(bb))) status = 7;
  if (status == 0 && bb == 0.0) {
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = 0.0;
  }
  bool done = status != 0 || bb == 0.0 || rr <= tol2;
  double alpha = (del > 0.0) ? gam / del : 0.0, beta = 0.0;
  double rgam = 0.0, ralpha = 0.0;
  cg_recips(gam, del, rgam, ralpha);
  if (!done && !(del > 0.0)) { status = 3; done = true; }
  while (!done) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      p[k] = u[k] + beta * p[k];
      q[k] = w[k] + beta * q[k];
      x[k] += alpha * p[k];
      r[k] -= alpha * q[k];
    }
    // SSOR phase 1 (red voxels only: the black ones are overwritten by phase 2 before
    // anyone reads them); the colour-sorted warps keep this branch uniform
    if (!a.ssor) {
      minv<D, double>(Mp, bd, r, u);
    } else if (is_red) {
      minv<D, double>(Mp, bd, r, u);
#pragma unroll
      for (int k = 0; k < D; ++k) u[k] *= omega;
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) u[k] = 0.0;   // defined for threads without a voxel
    }
    if (own) {
#pragma unroll
      for (int k = 0; k < D; ++k) a.u[(size_t)k * ld + n] = u[k];
    }
    if (a.ssor && !ssor_phases()) return;
    if (!bar()) return;
    if (!product(u, a.u, w)) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[0] += r[k] * u[k];
      v[1] += w[k] * u[k];
      v[2] += r[k] * r[k];
    }
    if (!grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    ++it;
    rr = tot[2];
    cg_scalar_step(sh, tot[0], tot[1], rr, tol2, it, a.max_iter, alpha, beta, gam, rgam, ralpha);
    const int code = sh.code;
    __syncthreads();
    if (code == 7) { status = 7; break; }
    if (code == 3) { status = 3; break; }
    if (code == 1) {
      // confirm with the true residual
      if (own) {
#pragma unroll
        for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
      }
      if (!bar()) return;
      if (!restart(tot)) return;
      gam = tot[0];
      del = tot[1];
      rr = tot[2];
      if (rr <= tol2) break;
      if (it >= a.max_iter) { status = 4; break; }
      ++restarts;
      alpha = del > 0.0 ? gam / del : 0.0;
      beta = 0.0;
      cg_recips(gam, del, rgam, ralpha);
#pragma unroll
      for (int k = 0; k < D; ++k) { p[k] = 0.0; q[k] = 0.0; }
      if (!(del > 0.0)) { status = 3; break; }
      continue;
    }
  }
  if (own) {
#pragma unroll
    for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
  }
  write_ctrl(a, it, restarts, rr, bb, rel0, status);
}

// ---------------------------------------------------------------------------------------
// Resident variant on the red-black reduced system. Eliminating the red voxels from
// B~ x = b (their rows read Dg_r x_r - scale .* sum of the black neighbours' x = b_r) leaves
// for the black voxels
//   S x_b = b^,   S = Dg_b - L Dg_r^-1 U,   b^ = b_b + scale .* sum_red nbrs Dg_r^-1 b_r,
// and afterwards x_r = Dg_r^-1 (b_r + scale .* sum of the black neighbours' x_b) (L, U:
// the couplings -scale between red and black neighbours; Dg: the voxel blocks
// B_n + diag(scale) deg_n with factor mfac). CG on S preconditioned by Dg_b takes the
// iterates of CG on B~ preconditioned by red-black symmetric Gauss-Seidel (SSOR with
// omega = 1): the two preconditioned operators share their spectrum apart from the
// eigenvalue 1 of the red unknowns. The residual of B~ at the recovered x equals the
// reduced residual (zero on the red rows), so the stop rule is unchanged; it is confirmed
// on B~ itself in FP64.
// One product with S is a red phase, y_r = Dg_r^-1 (scale .* sum of the black neighbours'
// u), and a black phase, w_b = Dg_b u_b - scale .* sum of the red neighbours' y; one plane
// array (a.u) carries u at the black voxels and y at the red ones. An iteration is the
// local update of the black voxels, two plain barriers and the reducing one (the SSOR form
// has four), and per pair of voxels three block solves and one block product (the SSOR
// form: four and two).
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(RB_MAX_THREADS, 1) k_pcg_rb(PcgArgs a) {
  extern __shared__ double smem[];
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  // per-slot edge weights in shared memory (read as broadcasts; no registers held)
  __shared__ double cwd[6];
  __shared__ float cwf[6];
  if (threadIdx.x == 0) {
    slot_weights(a, cwd);
    slot_weights(a, cwf);
  }
  __syncthreads();
  constexpr int NT = ntri(D);
  const int bd = blockDim.x, t = threadIdx.x;
  double* shB = smem;
  double* shM = smem + NT * bd;
  double* shH = smem + 2 * NT * bd;   // b^ (read at restarts only): shared, not registers
  int n = blockIdx.x * a.res_per + t;
  bool own = t < a.res_per && n < a.N;
  bool is_red = true;
  colour_sort(a, n, own, is_red);
  const bool red = own && is_red, black = own && !is_red;
  const size_t ld = a.ld;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const int e = tri(i, j);
      shB[e * bd + t] = own ? __ldg(a.blocks + (size_t)e * ld + n) : (i == j ? 1.0 : 0.0);
      shM[e * bd + t] = own ? __ldg(a.mfac + (size_t)e * ld + n) : (i == j ? 1.0 : 0.0);
    }
  int nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = (own && d < a.ndir) ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  const double degd = degree_of<double>(nb, cwd);
  // b is read from memory where it is needed (start, red recovery, true residual): the
  // black voxels' registers hold b^ instead
  // the prior scale is the same for every voxel: one shared copy instead of D registers
  __shared__ double s[RES_MAX_D];
  if (t < D) s[t] = __ldg(a.scale + t);
  __syncthreads();
  double x[D], r[D], u[D], w[D], p[D], q[D];
  auto load_b = [&](double* bv) {
#pragma unroll
    for (int k = 0; k < D; ++k) bv[k] = own ? __ldg(a.b + (size_t)k * ld + n) : 0.0;
  };
#pragma unroll
  for (int k = 0; k < D; ++k) {
    x[k] = own ? a.x[(size_t)k * ld + n] : 0.0;
    shH[k * bd + t] = 0.0;
    r[k] = 0.0;
    u[k] = 0.0;
    w[k] = 0.0;
    p[k] = 0.0;
    q[k] = 0.0;
  }
  const double* Bp = shB + t;
  const double* Mp = shM + t;
  double* U = a.u;
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  auto publish = [&](const double* v) {
#pragma unroll
    for (int k = 0; k < D; ++k) U[(size_t)k * ld + n] = v[k];
  };
  // red voxel: out = Dg^-1 (c + scale .* sum of the neighbours' U), c = 0 or b_r
  auto red_solve = [&](const double* c, double* out) {
    double sum[D], tv[D];
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (nb[d] >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += cwd[d] * ldx(U + (size_t)k * ld + nb[d]);
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) tv[k] = (c ? c[k] : 0.0) + s[k] * sum[k];
    minv<D, double>(Mp, bd, tv, out);
  };
  // out = S v on the black voxels (v in their registers); two barriers
  auto apply_S = [&](const double* v, double* out) -> bool {
    if (black) publish(v);
    if (!bar()) return false;
    if (red) {
      double y[D];
      red_solve(nullptr, y);
      publish(y);
    }
    if (!bar()) return false;
    if (black) amul<D, double>(Bp, bd, s, nb, cwd, degd, v, U, ld, out);
    return true;
  };
  // red voxels: x_r from the black voxels' x (one barrier); then every voxel's x is final
  auto recover_red = [&]() -> bool {
    if (black) publish(x);
    if (!bar()) return false;
    if (red) {
      double bv[D];
      load_b(bv);
      red_solve(bv, x);
    }
    return true;
  };
  // (r, u, w) of the reduced system from the current x_b, with partials (r'u, w'u, r'r, b'b)
  auto restart = [&](double* tot) -> bool {
    double bv[D];
    double sx[D];
    if (!apply_S(x, sx)) return false;
    if (black) {
#pragma unroll
      for (int k = 0; k < D; ++k) r[k] = shH[k * bd + t] - sx[k];
      minv<D, double>(Mp, bd, r, u);
    }
    if (!apply_S(u, w)) return false;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (black) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[0] += r[k] * u[k];
        v[1] += w[k] * u[k];
        v[2] += r[k] * r[k];
      }
    }
    load_b(bv);
#pragma unroll
    for (int k = 0; k < D; ++k) v[3] += bv[k] * bv[k];
    return grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };
  // ||b - B~ x||^2 of the full system at the current x (every voxel's x final), FP64
  auto true_residual = [&](double* tot) -> bool {
    if (own) {
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
    }
    if (!bar()) return false;
    double ax[D], bv[D], v[4] = {0.0, 0.0, 0.0, 0.0};
    if (own) {
      load_b(bv);
      amul<D, double>(Bp, bd, s, nb, cwd, degd, x, a.x, ld, ax);
#pragma unroll
      for (int k = 0; k < D; ++k) v[2] += (bv[k] - ax[k]) * (bv[k] - ax[k]);
    }
    return grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };

  // b^ = b_b + scale .* sum of the red neighbours' Dg_r^-1 b_r
  if (red) {
    double y[D], bv[D];
    load_b(bv);
    minv<D, double>(Mp, bd, bv, y);
    publish(y);
  }
  if (!bar()) return;
  if (black) {
    double sum[D];
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (nb[d] >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += cwd[d] * ldx(U + (size_t)k * ld + nb[d]);
      }
    }
    double bv[D];
    load_b(bv);
#pragma unroll
    for (int k = 0; k < D; ++k) shH[k * bd + t] = bv[k] + s[k] * sum[k];
  }
  double tot[4];
  if (!restart(tot)) return;   // (apply_S's first barrier orders the reads of U above)
  double gam = tot[0], del = tot[1], rr = tot[2];
  const double bb = tot[3];
  const double tol2 = a.delta * a.delta * bb;
  const double rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  int it = 0, restarts = 0, status = 0;
  bool x_final = false;   // the red voxels' x matches the current x_b
  if (!(isfinite(gam) && isfinite(del) && isfinite(bb))) status = 7;
  if (status == 0 && bb == 0.0) {
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = 0.0;
    x_final = true;
  }
  bool done = status != 0 || bb == 0.0;
  if (!done && rr <= tol2) {
    // the start value may already satisfy the tolerance: confirm on B~
    if (!recover_red()) return;
    if (!true_residual(tot)) return;
    x_final = true;
    rr = tot[2];
    done = rr <= tol2;
  }
  double alpha = (del > 0.0) ? gam / del : 0.0, beta = 0.0;
  double rgam = 0.0, ralpha = 0.0;
  cg_recips(gam, del, rgam, ralpha);
  if (!done && !(del > 0.0)) { status = 3; done = true; }
  while (!done) {
    if (black) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        p[k] = u[k] + beta * p[k];
        q[k] = w[k] + beta * q[k];
        x[k] += alpha * p[k];
        r[k] -= alpha * q[k];
      }
      minv<D, double>(Mp, bd, r, u);
    }
    x_final = false;
    if (!apply_S(u, w)) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (black) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[0] += r[k] * u[k];
        v[1] += w[k] * u[k];
        v[2] += r[k] * r[k];
      }
    }
    if (!grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    ++it;
    rr = tot[2];
    cg_scalar_step(sh, tot[0], tot[1], rr, tol2, it, a.max_iter, alpha, beta, gam, rgam, ralpha);
    const int code = sh.code;
    __syncthreads();
    if (code == 7) { status = 7; break; }
    if (code == 3) { status = 3; break; }
    if (code == 1) {
      // confirm with the true residual of B~
      if (!recover_red()) return;
      if (!true_residual(tot)) return;
      x_final = true;
      rr = tot[2];
      if (rr <= tol2) break;
      if (it >= a.max_iter) { status = 4; break; }
      ++restarts;
      if (!restart(tot)) return;
      gam = tot[0];
      del = tot[1];
      alpha = del > 0.0 ? gam / del : 0.0;
      beta = 0.0;
      cg_recips(gam, del, rgam, ralpha);
#pragma unroll
      for (int k = 0; k < D; ++k) { p[k] = 0.0; q[k] = 0.0; }
      if (!(del > 0.0)) { status = 3; break; }
      continue;
    }
  }
  if (!x_final && !recover_red()) return;
  if (own) {
#pragma unroll
    for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
  }
  write_ctrl(a, it, restarts, rr, bb, rel0, status);
}

// ---------------------------------------------------------------------------------------
// Streaming variant: same recurrence, vectors in global memory (x, r, u, w, p, s planes).
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_stream(PcgArgs a) {
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  // per-slot edge weights in shared memory (read as broadcasts; no registers held)
  __shared__ double cwd[6];
  __shared__ float cwf[6];
  // anisotropic prior: scale3[d][k] per direction and component
  __shared__ double s3[3][DMAX];
  if (threadIdx.x == 0) {
    slot_weights(a, cwd);
    slot_weights(a, cwf);
  }
  if (a.scale3 && threadIdx.x < 3 * D) s3[threadIdx.x / D][threadIdx.x % D] = a.scale3[threadIdx.x];
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const size_t ld = a.ld;
  const bool pre = a.mfac != nullptr;
  double s[D];
#pragma unroll
  for (int k = 0; k < D; ++k) s[k] = a.scale3 ? 0.0 : __ldg(a.scale + k);
  double* R = a.r;
  double* U = a.u;
  double* Wv = a.w;
  double* Pv = a.p;
  double* Sv = a.s;
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  auto load_nb = [&](int n, int* nb) {
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = d < a.ndir ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  };
  // edge weights of voxel n's slots: the direction weights, times the per-edge factors when
  // set (stored at each edge's lower voxel: n for +d, the neighbour for -d)
  auto weights_at = [&](int n, const int* nb, double* c6) {
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      c6[d] = cwd[d];
      if (a.ce && nb[d] >= 0)
        c6[d] *= (double)__uint_as_float((unsigned)__ldg(a.ce + (size_t)(d >> 1) * ld + ((d & 1) ? n : nb[d])) << 16);
    }
  };
  // (B~ v)_n with v_n = vn and the vector V for the neighbours
  auto product = [&](int n, const int* nb, const double* c6, const double* vn, const double* V,
                     double* out) {
    if (a.scale3) amul_dir<D>(a.blocks + n, (int)ld, s3, nb, c6, vn, V, ld, out);
    else amul<D, double>(a.blocks + n, (int)ld, s, nb, c6, degree_of<double>(nb, c6), vn, V, ld, out);
  };
  auto precond = [&](int n, const double* rn, double* un) {
    if (pre) {
      minv<D, double>(a.mfac + n, (int)ld, rn, un);
      if (a.ssor) {
#pragma unroll
        for (int k = 0; k < D; ++k) un[k] *= a.omega;   // SSOR phase 1
      }
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) un[k] = rn[k];
    }
  };
  // SSOR phases 2 (black voxels) and 3 (red voxels), each after a barrier
  auto ssor_rest = [&]() -> bool {
    if (!bar()) return false;
    for (int i = tid; i < a.n_black; i += nth) ssor_phase<D, double>(a, s, a.mfac, a.r, a.u, a.black[i], 2);
    if (!bar()) return false;
    for (int i = tid; i < a.n_red; i += nth) ssor_phase<D, double>(a, s, a.mfac, a.r, a.u, a.red[i], 3);
    return true;
  };
  // r = b - B~ x, u = M^-1 r (published); then w = B~ u and partials.
  auto restart = [&](double* tot) -> bool {
    for (int n = tid; n < a.N; n += nth) {
      int nb[6];
      load_nb(n, nb);
      double xn[D], ax[D], rn[D], un[D];
#pragma unroll
      for (int k = 0; k < D; ++k) xn[k] = ldx(a.x + (size_t)k * ld + n);
      double c6[6];
      weights_at(n, nb, c6);
      product(n, nb, c6, xn, a.x, ax);
#pragma unroll
      for (int k = 0; k < D; ++k) rn[k] = __ldg(a.b + (size_t)k * ld + n) - ax[k];
      precond(n, rn, un);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        R[(size_t)k * ld + n] = rn[k];
        U[(size_t)k * ld + n] = un[k];
        Pv[(size_t)k * ld + n] = 0.0;
        Sv[(size_t)k * ld + n] = 0.0;
      }
    }
    if (a.ssor && !ssor_rest()) return false;
    if (!bar()) return false;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = tid; n < a.N; n += nth) {
      int nb[6];
      load_nb(n, nb);
      double un[D], wn[D];
#pragma unroll
      for (int k = 0; k < D; ++k) un[k] = U[(size_t)k * ld + n];
      double c6[6];
      weights_at(n, nb, c6);
      product(n, nb, c6, un, U, wn);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double rk = R[(size_t)k * ld + n], bk = __ldg(a.b + (size_t)k * ld + n);
        Wv[(size_t)k * ld + n] = wn[k];
        v[0] += rk * un[k];
        v[1] += wn[k] * un[k];
        v[2] += rk * rk;
        v[3] += bk * bk;
      }
    }
    return grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };

  double tot[4];
  if (!restart(tot)) return;
  double gam = tot[0], del = tot[1], rr = tot[2];
  const double bb = tot[3];
  const double tol2 = a.delta * a.delta * bb;
  const double rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  int it = 0, restarts = 0, status = 0;
  if (!(isfinite(gam) && isfinite(del) && isfinite(bb))) status = 7;
  if (status == 0 && bb == 0.0) {
    for (int n = tid; n < a.N; n += nth)
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = 0.0;
  }
  bool done = status != 0 || bb == 0.0 || rr <= tol2;
  double alpha = (del > 0.0) ? gam / del : 0.0, beta = 0.0;
  double rgam = 0.0, ralpha = 0.0;
  cg_recips(gam, del, rgam, ralpha);
  if (!done && !(del > 0.0)) { status = 3; done = true; }
  while (!done) {
    for (int n = tid; n < a.N; n += nth) {
      // all loads first (the compiler cannot prove the vectors distinct)
      double rn[D], un[D], pk[D], sk[D], xk[D], wk[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * ld + n;
        un[k] = U[o];
        pk[k] = Pv[o];
        wk[k] = Wv[o];
        sk[k] = Sv[o];
        xk[k] = a.x[o];
        rn[k] = R[o];
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        pk[k] = un[k] + beta * pk[k];
        sk[k] = wk[k] + beta * sk[k];
        xk[k] += alpha * pk[k];
        rn[k] -= alpha * sk[k];
      }
      precond(n, rn, un);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * ld + n;
        Pv[o] = pk[k];
        Sv[o] = sk[k];
        a.x[o] = xk[k];
        R[o] = rn[k];
        U[o] = un[k];
      }
    }
    if (a.ssor && !ssor_rest()) return;
    if (!bar()) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = tid; n < a.N; n += nth) {
      int nb[6];
      load_nb(n, nb);
      double un[D], wn[D], rk[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        un[k] = U[(size_t)k * ld + n];
        rk[k] = R[(size_t)k * ld + n];
      }
      double c6[6];
      weights_at(n, nb, c6);
      product(n, nb, c6, un, U, wn);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[0] += rk[k] * un[k];
        v[1] += wn[k] * un[k];
        v[2] += rk[k] * rk[k];
      }
#pragma unroll
      for (int k = 0; k < D; ++k) Wv[(size_t)k * ld + n] = wn[k];
    }
    if (!grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    ++it;
    rr = tot[2];
    cg_scalar_step(sh, tot[0], tot[1], rr, tol2, it, a.max_iter, alpha, beta, gam, rgam, ralpha);
    const int code = sh.code;
    __syncthreads();
    if (code == 7) { status = 7; break; }
    if (code == 3) { status = 3; break; }
    if (code == 1) {
      // x was last updated before the reducing barrier above, so it is complete
      if (!restart(tot)) return;
      gam = tot[0];
      del = tot[1];
      rr = tot[2];
      if (rr <= tol2) break;
      if (it >= a.max_iter) { status = 4; break; }
      ++restarts;
      alpha = del > 0.0 ? gam / del : 0.0;
      beta = 0.0;
      cg_recips(gam, del, rgam, ralpha);
      if (!(del > 0.0)) { status = 3; break; }
      continue;
    }
  }
  write_ctrl(a, it, restarts, rr, bb, rel0, status);
}


// ---------------------------------------------------------------------------------------
// The L'L prior (D_w = L'L): the streaming recurrence of k_pcg_stream with a two-pass
// operator. A product B~ v first forms t = L v over every voxel, then, after a grid barrier,
// (B~ v)_n = B_n v_n + scale .* (L t)_n: each product costs one more barrier, and its stencil
// reaches the neighbours' neighbours (25 points in 3D) through t. Block-Jacobi (blocks plus
// diag(scale) times the diagonal of L'L) or no preconditioner.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_ltl(PcgArgs a) {
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  __shared__ double cwd[6];
  if (threadIdx.x == 0) slot_weights(a, cwd);
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const size_t ld = a.ld;
  const bool pre = a.mfac != nullptr;
  double s[D];
#pragma unroll
  for (int k = 0; k < D; ++k) s[k] = __ldg(a.scale + k);
  double* R = a.r;
  double* U = a.u;
  double* Wv = a.w;
  double* Pv = a.p;
  double* Sv = a.s;
  double* Tv = a.t;
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  // sum_m c_m V[m] over the in-mask neighbours of n, and the weighted degree
  auto nsum = [&](int n, const double* V, double* sum) -> double {
    double deg = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const int m = d < a.ndir ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
      if (m >= 0) {
        deg += cwd[d];
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += cwd[d] * ldx(V + (size_t)k * ld + m);
      }
    }
    return deg;
  };
  // pass 1 of a product: t = L V for every voxel (V complete: a barrier precedes)
  auto lap_pass = [&](const double* V) {
    for (int n = tid; n < a.N; n += nth) {
      double sum[D];
      const double deg = nsum(n, V, sum);
#pragma unroll
      for (int k = 0; k < D; ++k) Tv[(size_t)k * ld + n] = deg * ldx(V + (size_t)k * ld + n) - sum[k];
    }
  };
  // pass 2 at voxel n: out = B_n v + scale .* (L t)_n (t complete: a barrier precedes)
  auto op_at = [&](int n, const double* v, double* out) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) acc += __ldg(a.blocks + (size_t)(i >= j ? tri(i, j) : tri(j, i)) * ld + n) * v[j];
      out[i] = acc;
    }
    double sum[D];
    const double deg = nsum(n, Tv, sum);
#pragma unroll
    for (int k = 0; k < D; ++k) out[k] += s[k] * (deg * ldx(Tv + (size_t)k * ld + n) - sum[k]);
  };
  auto precond = [&](int n, const double* rn, double* un) {
    if (pre) {
      minv<D, double>(a.mfac + n, (int)ld, rn, un);
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) un[k] = rn[k];
    }
  };
  // r = b - B~ x, u = M^-1 r (published); then w = B~ u and the partials
  auto restart = [&](double* tot) -> bool {
    lap_pass(a.x);
    if (!bar()) return false;
    for (int n = tid; n < a.N; n += nth) {
      double xn[D], ax[D], rn[D], un[D];
#pragma unroll
      for (int k = 0; k < D; ++k) xn[k] = ldx(a.x + (size_t)k * ld + n);
      op_at(n, xn, ax);
#pragma unroll
      for (int k = 0; k < D; ++k) rn[k] = __ldg(a.b + (size_t)k * ld + n) - ax[k];
      precond(n, rn, un);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        R[(size_t)k * ld + n] = rn[k];
        U[(size_t)k * ld + n] = un[k];
        Pv[(size_t)k * ld + n] = 0.0;
        Sv[(size_t)k * ld + n] = 0.0;
      }
    }
    if (!bar()) return false;
    lap_pass(U);
    if (!bar()) return false;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = tid; n < a.N; n += nth) {
      double un[D], wn[D];
#pragma unroll
      for (int k = 0; k < D; ++k) un[k] = U[(size_t)k * ld + n];
      op_at(n, un, wn);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double rk = R[(size_t)k * ld + n], bk = __ldg(a.b + (size_t)k * ld + n);
        Wv[(size_t)k * ld + n] = wn[k];
        v[0] += rk * un[k];
        v[1] += wn[k] * un[k];
        v[2] += rk * rk;
        v[3] += bk * bk;
      }
    }
    return grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };

  double tot[4];
  if (!restart(tot)) return;
  double gam = tot[0], del = tot[1], rr = tot[2];
  const double bb = tot[3];
  const double tol2 = a.delta * a.delta * bb;
  const double rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  int it = 0, restarts = 0, status = 0;
  if (!(isfinite(gam) && isfinite(del) && isfinite(bb))) status = 7;
  if (status == 0 && bb == 0.0) {
    for (int n = tid; n < a.N; n += nth)
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = 0.0;
  }
  bool done = status != 0 || bb == 0.0 || rr <= tol2;
  double alpha = (del > 0.0) ? gam / del : 0.0, beta = 0.0;
  double rgam = 0.0, ralpha = 0.0;
  cg_recips(gam, del, rgam, ralpha);
  if (!done && !(del > 0.0)) { status = 3; done = true; }
  while (!done) {
    for (int n = tid; n < a.N; n += nth) {
      double rn[D], un[D], pk[D], sk[D], xk[D], wk[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * ld + n;
        un[k] = U[o];
        pk[k] = Pv[o];
        wk[k] = Wv[o];
        sk[k] = Sv[o];
        xk[k] = a.x[o];
        rn[k] = R[o];
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        pk[k] = un[k] + beta * pk[k];
        sk[k] = wk[k] + beta * sk[k];
        xk[k] += alpha * pk[k];
        rn[k] -= alpha * sk[k];
      }
      precond(n, rn, un);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * ld + n;
        Pv[o] = pk[k];
        Sv[o] = sk[k];
        a.x[o] = xk[k];
        R[o] = rn[k];
        U[o] = un[k];
      }
    }
    if (!bar()) return;
    lap_pass(U);
    if (!bar()) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = tid; n < a.N; n += nth) {
      double un[D], wn[D], rk[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        un[k] = U[(size_t)k * ld + n];
        rk[k] = R[(size_t)k * ld + n];
      }
      op_at(n, un, wn);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[0] += rk[k] * un[k];
        v[1] += wn[k] * un[k];
        v[2] += rk[k] * rk[k];
        Wv[(size_t)k * ld + n] = wn[k];
      }
    }
    if (!grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    ++it;
    rr = tot[2];
    cg_scalar_step(sh, tot[0], tot[1], rr, tol2, it, a.max_iter, alpha, beta, gam, rgam, ralpha);
    const int code = sh.code;
    __syncthreads();
    if (code == 7) { status = 7; break; }
    if (code == 3) { status = 3; break; }
    if (code == 1) {
      // x was last updated before the reducing barrier above, so it is complete
      if (!restart(tot)) return;
      gam = tot[0];
      del = tot[1];
      rr = tot[2];
      if (rr <= tol2) break;
      if (it >= a.max_iter) { status = 4; break; }
      ++restarts;
      alpha = del > 0.0 ? gam / del : 0.0;
      beta = 0.0;
      cg_recips(gam, del, rgam, ralpha);
      if (!(del > 0.0)) { status = 3; break; }
      continue;
    }
  }
  write_ctrl(a, it, restarts, rr, bb, rel0, status);
}

// ---------------------------------------------------------------------------------------
// Mixed precision (resident): FP64 iterative refinement around FP32 CG-CG inner solves.
//   outer: r = b - B~ x (FP64 blocks, FP64 arithmetic), stop when ||r|| <= delta ||b||;
//   inner: B~ d = r in FP32 (FP32 blocks, preconditioner and vectors) to ||r_in|| <=
//          inner_tol ||r||, then x += d in FP64.
// Per-thread inner-product terms are formed in FP32 over the voxel's D components and
// accumulated across threads and CTAs in FP64 (fixed order).
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(RES_MAX_THREADS, 1) k_pcg_mixed_res(PcgArgs a) {
  extern __shared__ double smem[];
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  // per-slot edge weights in shared memory (read as broadcasts; no registers held)
  __shared__ double cwd[6];
  __shared__ float cwf[6];
  if (threadIdx.x == 0) {
    slot_weights(a, cwd);
    slot_weights(a, cwf);
  }
  __syncthreads();
  constexpr int NT = ntri(D);
  const int bd = blockDim.x, t = threadIdx.x;
  double* shB = smem;                                   // [NT][bd] FP64 blocks
  float* shB32 = reinterpret_cast<float*>(smem + NT * bd);   // [NT][bd]
  float* shM32 = shB32 + NT * bd;                       // [NT][bd]
  int n = blockIdx.x * a.res_per + t;
  bool own = t < a.res_per && n < a.N;
  bool is_red = true;
  if (a.ssor) colour_sort(a, n, own, is_red);
  const size_t ld = a.ld;
  const bool pre = a.mfac32 != nullptr;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const int e = tri(i, j);
      shB[e * bd + t] = own ? __ldg(a.blocks + (size_t)e * ld + n) : (i == j ? 1.0 : 0.0);
      shB32[e * bd + t] = own ? __ldg(a.blocks32 + (size_t)e * ld + n) : (i == j ? 1.f : 0.f);
      shM32[e * bd + t] = (own && pre) ? __ldg(a.mfac32 + (size_t)e * ld + n) : (i == j ? 1.f : 0.f);
    }
  int nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = (own && d < a.ndir) ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  const double degd = degree_of<double>(nb, cwd);
  const float degf = (float)degd;
  double s[D], x[D], bv[D];
  float s32[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    s[k] = __ldg(a.scale + k);
    s32[k] = (float)s[k];
    x[k] = own ? a.x[(size_t)k * ld + n] : 0.0;
    bv[k] = own ? __ldg(a.b + (size_t)k * ld + n) : 0.0;
  }
  const double* Bp = shB + t;
  const float* Bp32 = shB32 + t;
  const float* Mp32 = shM32 + t;
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  double tot[4];
  int outer = 0, inner_total = 0, status = 0;
  double bb = 0.0, rr = 0.0, rel0 = 0.0, tol2 = 0.0;
  while (true) {
    // ---- FP64 true residual (x of every voxel is complete: start value or published) ----
    double r64[D];
    {
      double ax[D];
      amul<D, double>(Bp, bd, s, nb, cwd, degd, x, a.x, ld, ax);
      double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < D; ++k) {
        r64[k] = bv[k] - ax[k];
        v[0] += r64[k] * r64[k];
        v[1] += bv[k] * bv[k];
      }
      if (!grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    }
    rr = tot[0];
    if (outer == 0) {
      bb = tot[1];
      tol2 = a.delta * a.delta * bb;
      rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      if (!(isfinite(rr) && isfinite(bb))) { status = 7; break; }
      if (bb == 0.0) {
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = 0.0;
        break;
      }
    }
    if (!isfinite(rr)) { status = 7; break; }
    if (rr <= tol2) break;
    if (inner_total >= a.max_iter) { status = 4; break; }
    ++outer;
    // ---- FP32 inner CG-CG on B~ d = r ----
    float r[D], u[D], w[D], p[D], q[D], d[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      r[k] = (float)r64[k];
      d[k] = 0.f;
      p[k] = 0.f;
      q[k] = 0.f;
    }
    // inner target: inner_tol relative, but no further than the outer stop needs
    const double itol2 = fmax(a.inner_tol * a.inner_tol * rr, 0.25 * tol2);
    if (!a.ssor) {
      minv<D, float>(Mp32, bd, r, u);
    } else if (is_red) {   // SSOR phase 1, red voxels only
      minv<D, float>(Mp32, bd, r, u);
#pragma unroll
      for (int k = 0; k < D; ++k) u[k] *= (float)a.omega;
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) u[k] = 0.f;   // defined for threads without a voxel
    }
    if (own) {
#pragma unroll
      for (int k = 0; k < D; ++k) a.u32[(size_t)k * ld + n] = u[k];
    }
    if (a.ssor && !resident_ssor_phases<D, float>(a, bar, own, is_red, nb, s32, Mp32, bd, n, r, u, a.u32))
      return;
    if (!bar()) return;
    amul<D, float>(Bp32, bd, s32, nb, cwf, degf, u, a.u32, ld, w);
    {
      float g = 0.f, dl = 0.f, q2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        g += r[k] * u[k];
        dl += w[k] * u[k];
        q2 += r[k] * r[k];
      }
      const FF v[4] = {ff_of(g), ff_of(dl), ff_of(q2), ff_of(0.f)};
      if (!grid_allreduce4_ff(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    }
    double gam = tot[0], del = tot[1];
    if (!(del > 0.0) || !isfinite(del)) { status = isfinite(del) ? 3 : 7; break; }
    double alpha = gam / del, beta = 0.0;
    double rgam = 0.0, ralpha = 0.0;
    cg_recips(gam, del, rgam, ralpha);
    int it = 0;
    while (true) {
      const float fa = (float)alpha, fb = (float)beta;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        p[k] = u[k] + fb * p[k];
        q[k] = w[k] + fb * q[k];
        d[k] += fa * p[k];
        r[k] -= fa * q[k];
      }
      if (!a.ssor) {
        minv<D, float>(Mp32, bd, r, u);
      } else if (is_red) {   // SSOR phase 1, red voxels only
        minv<D, float>(Mp32, bd, r, u);
#pragma unroll
        for (int k = 0; k < D; ++k) u[k] *= (float)a.omega;
      } else {
#pragma unroll
        for (int k = 0; k < D; ++k) u[k] = 0.f;   // defined for threads without a voxel
      }
      if (own) {
#pragma unroll
        for (int k = 0; k < D; ++k) a.u32[(size_t)k * ld + n] = u[k];
      }
      if (a.ssor && !resident_ssor_phases<D, float>(a, bar, own, is_red, nb, s32, Mp32, bd, n, r, u, a.u32))
        return;
      if (!bar()) return;
      amul<D, float>(Bp32, bd, s32, nb, cwf, degf, u, a.u32, ld, w);
      float g = 0.f, dl = 0.f, q2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        g += r[k] * u[k];
        dl += w[k] * u[k];
        q2 += r[k] * r[k];
      }
      const FF v[4] = {ff_of(g), ff_of(dl), ff_of(q2), ff_of(0.f)};
      if (!grid_allreduce4_ff(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
      ++it;
      const bool capped = it >= a.max_inner || inner_total + it >= a.max_iter;
      cg_scalar_step(sh, tot[0], tot[1], tot[2], itol2, capped ? 1 : 0, 1, alpha, beta, gam, rgam, ralpha);
      const int code = sh.code;
      __syncthreads();
      if (code == 7) { status = 7; break; }
      if (code != 0) break;   // inner tolerance, iteration cap, or loss of conjugacy in FP32
    }
    inner_total += it;
    if (status != 0) break;
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] += (double)d[k];
    if (own) {
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
    }
    if (!bar()) return;
  }
  if (own) {
#pragma unroll
    for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->iterations = inner_total;
    a.ctrl->restarts = outer;
    a.ctrl->rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    a.ctrl->rel_res0 = rel0;
    a.ctrl->status = status;
    if (status != 0 && a.ctrl->status_any == 0) a.ctrl->status_any = status;
    a.ctrl->iter_total += inner_total;
    a.ctrl->solves += 1;
  }
}

// ---------------------------------------------------------------------------------------
// Pipelined CG (Ghysels & Vanroose 2014) on the same reduced system, split-preconditioned:
// with Dg_b = L_b L_b' (the block-Jacobi factor of each black voxel), CG runs without a
// preconditioner on  S^ = L_b^-1 S L_b^-T = I - L_b^-1 L Dg_r^-1 U L_b^-T  in the variable
// x^ = L_b' x_b. Its iterates are those of CG on S preconditioned by Dg_b (the same Krylov
// spaces; r = L_b r^), but a product with S^ costs two triangular products at the black voxel
// and one block product at the red one, where the preconditioned form needs three full block
// products (M^-1, Dg_r^-1, Dg_b), and the recurrences for u = M^-1 r and q = M^-1 s go away.
// The two inner products of iteration i come from r^_i and w^_i = S^ r^_i before its product,
// so their reduction completes at the product's first barrier: two grid barriers per
// iteration. Per iteration (black voxels):
//   gamma = r^'r^, delta = w^'r^, rr = |L_b r^|^2 = |r|^2 (posted)   v = L_b^-T w^ (published)
//   --- barrier: the partials and v are visible --- red phase y = Dg_r^-1 (scale .* sum v);
//   every CTA sums the partials in a fixed order and forms alpha, beta (Chronopoulos & Gear)
//   --- barrier ---  n = w^ - L_b^-1 (scale .* sum y)  (= S^ w^)
//   z = n + beta z, s = w^ + beta s, p = r^ + beta p, x^ += alpha p, r^ -= alpha s,
//   w^ -= alpha z.
// The stop test reads the unscaled reduced residual |r| (= the black rows of B~'s residual
// once the red voxels are recovered) one product earlier than the unpipelined form; the stop
// is confirmed on B~'s true residual as in k_pcg_rb. p, s, z live in shared memory beside
// L_b and L_b^-1 (black voxels) or Dg_r^-1 (red voxels); the data blocks are read from global
// memory by the rare restart and confirmation passes only.
// ---------------------------------------------------------------------------------------
// PRIOR_SCALE3: the anisotropic prior's scales move into the neighbour sums (s = 1);
// PRIOR_EDGE: the voxel's six slot weights (per-edge factors) in shared memory after z.
template <int D, int PRIOR>
__global__ void __launch_bounds__(RB_MAX_THREADS, 1) k_pcg_rbp(PcgArgs a) {
  constexpr bool ANISO = PRIOR == PRIOR_SCALE3;
  extern __shared__ double smem[];
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  __shared__ double cwd[6];
  if (threadIdx.x == 0) slot_weights(a, cwd);
  __syncthreads();
  constexpr int NT = ntri(D);
  const int bd = blockDim.x, t = threadIdx.x;
  double* shL = smem;                 // black: L_b (true diagonal)
  double* shM = smem + NT * bd;       // black: L_b^-1; red: Dg_r^-1
  double* shH = smem + 2 * NT * bd;   // b^
  double* shP = shH + D * bd;         // p
  double* shS = shP + D * bd;         // s = S^ p
  double* shZ = shS + D * bd;         // z = S^ s
  int n = blockIdx.x * a.res_per + t;
  bool own = t < a.res_per && n < a.N;
  bool is_red = true;
  colour_sort(a, n, own, is_red);
  const bool red = own && is_red, black = own && !is_red;
  const size_t ld = a.ld;
  {
    double Lf[NT];
#pragma unroll
    for (int e = 0; e < NT; ++e) Lf[e] = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) Lf[tri(i, i)] = 1.0;
    if (own) {
#pragma unroll
      for (int e = 0; e < NT; ++e) Lf[e] = __ldg(a.mfac + (size_t)e * ld + n);
    }
#pragma unroll
    for (int e = 0; e < NT; ++e) shM[e * bd + t] = Lf[e];
    if (black) {
      // L_b with its true diagonal, and L_b^-1 in place of the factor
      double Li[NT];
      lower_inverse<D, double>(shM + t, bd, Li);
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          const int e = tri(i, j);
          shL[e * bd + t] = i == j ? 1.0 / Lf[e] : Lf[e];
          shM[e * bd + t] = Li[e];
        }
    } else {
      // red voxels (and threads without a voxel): the explicit inverse Dg_r^-1
      factor_to_inverse<D, double>(shM + t, bd);
    }
  }
  int nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = (own && d < a.ndir) ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  double* shC = shZ + D * bd;         // PRIOR_EDGE: slot weights [6][bd]
  if constexpr (PRIOR == PRIOR_EDGE) {
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      double c = cwd[d];
      // the edge's factor is stored at its lower voxel: n for +d, the neighbour for -d
      if (nb[d] >= 0)
        c *= (double)__uint_as_float((unsigned)__ldg(a.ce + (size_t)(d >> 1) * ld + ((d & 1) ? n : nb[d])) << 16);
      shC[d * bd + t] = c;
    }
  }
  __shared__ double s[RES_MAX_D];
  __shared__ double s3[ANISO ? 3 : 1][ANISO ? DMAX : 1];
  if (t < D) s[t] = ANISO ? 1.0 : __ldg(a.scale + t);
  if constexpr (ANISO) {
    if (t < 3 * D) s3[t / D][t % D] = a.scale3[t];
  }
  __syncthreads();
  double x[D], r[D], w[D];   // x holds x_b outside the iteration, x^ inside it
  auto load_b = [&](double* bv) {
#pragma unroll
    for (int k = 0; k < D; ++k) bv[k] = own ? __ldg(a.b + (size_t)k * ld + n) : 0.0;
  };
#pragma unroll
  for (int k = 0; k < D; ++k) {
    x[k] = own ? a.x[(size_t)k * ld + n] : 0.0;
    r[k] = w[k] = 0.0;
    shH[k * bd + t] = 0.0;
  }
  const double* Lp = shL + t;
  const double* Mp = shM + t;
  const double* Bg = a.blocks + n;     // data block in global memory (own voxels only)
  double* U = a.u;
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  auto publish = [&](const double* v) {
#pragma unroll
    for (int k = 0; k < D; ++k) U[(size_t)k * ld + n] = v[k];
  };
  auto nsum = [&](double* sum) {
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (nb[d] >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          if constexpr (ANISO) sum[k] += s3[d >> 1][k] * cwd[d] * ldx(U + (size_t)k * ld + nb[d]);
          else if constexpr (PRIOR == PRIOR_EDGE) sum[k] += shC[d * bd + t] * ldx(U + (size_t)k * ld + nb[d]);
          else sum[k] += cwd[d] * ldx(U + (size_t)k * ld + nb[d]);
        }
      }
    }
  };
  auto red_solve = [&](const double* c, double* out) {
    double sum[D], tv[D];
    nsum(sum);
#pragma unroll
    for (int k = 0; k < D; ++k) tv[k] = (c ? c[k] : 0.0) + s[k] * sum[k];
    symv<D, double>(Mp, bd, tv, out);
  };
  // out = S^ v at the black voxels: v' = L_b^-T v published, red phase, then
  // out = v - L_b^-1 (scale .* sum of the red neighbours' y)
  auto apply_Sh = [&](const double* v, double* out) -> bool {
    if (black) {
      double vt[D];
      trmv<D, double, false>(Mp, bd, v, vt);
      publish(vt);
    }
    if (!bar()) return false;
    if (red) {
      double y[D];
      red_solve(nullptr, y);
      publish(y);
    }
    if (!bar()) return false;
    if (black) {
      double sum[D], tv[D];
      nsum(sum);
#pragma unroll
      for (int k = 0; k < D; ++k) tv[k] = s[k] * sum[k];
      trmv<D, double, true>(Mp, bd, tv, out);
#pragma unroll
      for (int k = 0; k < D; ++k) out[k] = v[k] - out[k];
    }
    return true;
  };
  // out = S v at the black voxels in unscaled variables (restarts only)
  auto apply_S = [&](const double* v, double* out) -> bool {
    if (black) publish(v);
    if (!bar()) return false;
    if (red) {
      double y[D];
      red_solve(nullptr, y);
      publish(y);
    }
    if (!bar()) return false;
    if (black) {
      if constexpr (ANISO) {
        amul_dir<D>(Bg, (int)ld, s3, nb, cwd, v, U, ld, out);
      } else if constexpr (PRIOR == PRIOR_EDGE) {
        double c6[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) c6[d] = shC[d * bd + t];
        const double degd = degree_of<double>(nb, c6);
        amul<D, double>(Bg, (int)ld, s, nb, c6, degd, v, U, ld, out);
      } else {
        const double degd = degree_of<double>(nb, cwd);
        amul<D, double>(Bg, (int)ld, s, nb, cwd, degd, v, U, ld, out);
      }
    }
    return true;
  };
  // x_b = L_b^-T x^, then the red voxels from their rows
  auto recover_red = [&]() -> bool {
    if (black) {
      double xb[D];
      trmv<D, double, false>(Mp, bd, x, xb);
#pragma unroll
      for (int k = 0; k < D; ++k) x[k] = xb[k];
      publish(x);
    }
    if (!bar()) return false;
    if (red) {
      double bv[D];
      load_b(bv);
      red_solve(bv, x);
    }
    return true;
  };
  auto true_residual = [&](double* tot) -> bool {
    if (own) {
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
    }
    if (!bar()) return false;
    double ax[D], bv[D], v[4] = {0.0, 0.0, 0.0, 0.0};
    if (own) {
      load_b(bv);
      if constexpr (ANISO) {
        amul_dir<D>(Bg, (int)ld, s3, nb, cwd, x, a.x, ld, ax);
      } else if constexpr (PRIOR == PRIOR_EDGE) {
        double c6[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) c6[d] = shC[d * bd + t];
        const double degd = degree_of<double>(nb, c6);
        amul<D, double>(Bg, (int)ld, s, nb, c6, degd, x, a.x, ld, ax);
      } else {
        const double degd = degree_of<double>(nb, cwd);
        amul<D, double>(Bg, (int)ld, s, nb, cwd, degd, x, a.x, ld, ax);
      }
#pragma unroll
      for (int k = 0; k < D; ++k) v[2] += (bv[k] - ax[k]) * (bv[k] - ax[k]);
    }
    return grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };
  // (re)start of the recurrences from the current x_b: r^ = L_b^-1 (b^ - S x_b),
  // x^ = L_b' x_b, w^ = S^ r^, p = s = z = 0
  auto restart = [&]() -> bool {
    double sx[D];
    if (!apply_S(x, sx)) return false;
    if (black) {
      double rb[D], xh[D];
#pragma unroll
      for (int k = 0; k < D; ++k) rb[k] = shH[k * bd + t] - sx[k];
      trmv<D, double, true>(Mp, bd, rb, r);
      trmv<D, double, false>(Lp, bd, x, xh);
#pragma unroll
      for (int k = 0; k < D; ++k) x[k] = xh[k];
    }
    if (!apply_Sh(r, w)) return false;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      shP[k * bd + t] = 0.0;
      shS[k * bd + t] = 0.0;
      shZ[k * bd + t] = 0.0;
    }
    return true;
  };

  // b^ = b_b + scale .* sum of the red neighbours' Dg_r^-1 b_r
  if (red) {
    double y[D], bv[D];
    load_b(bv);
    symv<D, double>(Mp, bd, bv, y);
    publish(y);
  }
  if (!bar()) return;
  if (black) {
    double sum[D], bv[D];
    nsum(sum);
    load_b(bv);
#pragma unroll
    for (int k = 0; k < D; ++k) shH[k * bd + t] = bv[k] + s[k] * sum[k];
  }
  if (!restart()) return;   // (apply_S's first barrier orders the reads of U above)
  double tot[4];
  double bb = 0.0, tol2 = 0.0, rel0 = 0.0, rr = 0.0;
  double alpha = 0.0, beta = 0.0, gam = 0.0, rgam = 0.0, ralpha = 0.0;
  int it = 0, restarts = 0, status = 0;
  bool first = true;        // first pass of the solve: the partials carry b'b
  bool x_final = false;     // x holds x_b (and the red voxels are recovered)
  while (true) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (black) {
      // v = L_b^-T w^ first, so that its stores are in flight during the block reduction
      double vt[D], lr[D];
      trmv<D, double, false>(Mp, bd, w, vt);
      publish(vt);
      trmv<D, double, true>(Lp, bd, r, lr);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[0] += r[k] * r[k];
        v[1] += w[k] * r[k];
        v[2] += lr[k] * lr[k];
      }
    }
    if (first) {
      double bv[D];
      load_b(bv);
#pragma unroll
      for (int k = 0; k < D; ++k) v[3] += bv[k] * bv[k];
    }
    const double* part = allreduce4_post(a.part, a.part1, v, sh.red);
    if (!bar()) return;                 // partials and v are visible everywhere
    if (red) {
      double y[D];
      red_solve(nullptr, y);
      publish(y);
    }
    // before the next barrier; the loads run on the last four warps (black voxels or none,
    // idle in the red phase), beside the red warps' neighbour loads
    allreduce4_collect(part, sh.red, tot, bd >= 128 ? (bd >> 5) - 4 : 0);
    if (first) {
      bb = tot[3];
      tol2 = a.delta * a.delta * bb;
      rel0 = bb > 0.0 ? sqrt(tot[2] / bb) : 0.0;
      first = false;
      if (!(isfinite(tot[0]) && isfinite(tot[1]) && isfinite(bb))) status = 7;
    }
    rr = tot[2];
    if (status == 0 && bb == 0.0) {
#pragma unroll
      for (int k = 0; k < D; ++k) x[k] = 0.0;
      x_final = true;
    }
    int code = 0;
    if (status == 0 && bb != 0.0) {
      cg_scalar_step(sh, tot[0], tot[1], rr, tol2, it, a.max_iter, alpha, beta, gam, rgam, ralpha);
      code = sh.code;
      __syncthreads();
    }
    if (!bar()) return;                 // the red phase's y is visible; all partials read
    if (status != 0 || bb == 0.0) break;
    if (code == 7) { status = 7; break; }
    if (code == 3) { status = 3; break; }
    if (code == 1) {
      // confirm with the true residual of B~
      if (!recover_red()) return;
      if (!true_residual(tot)) return;
      x_final = true;
      rr = tot[2];
      if (rr <= tol2) break;
      if (it >= a.max_iter) { status = 4; break; }
      ++restarts;
      if (!restart()) return;
      x_final = false;
      rgam = 0.0;
      ralpha = 0.0;
      continue;
    }
    if (black) {
      double sum[D], tv[D], nn[D];
      nsum(sum);
#pragma unroll
      for (int k = 0; k < D; ++k) tv[k] = s[k] * sum[k];
      trmv<D, double, true>(Mp, bd, tv, nn);   // n = w^ - L_b^-1 (scale .* sum y)
      const double al = alpha, be = beta;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int o = k * bd + t;
        const double z = (w[k] - nn[k]) + be * shZ[o];
        const double sv = w[k] + be * shS[o];
        const double p = r[k] + be * shP[o];
        shZ[o] = z;
        shS[o] = sv;
        shP[o] = p;
        x[k] += al * p;
        r[k] -= al * sv;
        w[k] -= al * z;
      }
    }
    ++it;
  }
  if (!x_final && !recover_red()) return;
  if (own) {
#pragma unroll
    for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
  }
  write_ctrl(a, it, restarts, rr, bb, rel0, status);
}

// ---------------------------------------------------------------------------------------
// The pipelined reduced solver on lane pairs (k_pcg_rbp2): the iteration of k_pcg_rbp, with
// the CTA's red and black voxels paired up. Lanes 2q and 2q + 1 of the CTA hold red voxel q
// and black voxel q of the CTA together, and lane h of the pair owns the components
// k = 2j + h of both. In k_pcg_rbp one thread holds one voxel, so only the threads of one
// colour work in each phase and half the warps idle; here every lane works in every phase,
// on half of a voxel of the phase's colour, so each phase has twice the independent FP64
// chains in flight with the same number of threads. Products with a block (triangular or
// symmetric) are split by rows: both lanes gather the whole input vector (one __shfl_xor per
// component) and form their own rows; neighbour sums, vector updates and inner-product
// partials are split by components. Both lanes of a pair take the same branches, and every
// gather runs where the whole warp takes part.
// ---------------------------------------------------------------------------------------
namespace {

constexpr int RB2_MAX_THREADS = 384;   // two lanes per slot; 12 warps leave 168 registers

// full[D] from this lane's components (2j + h) and its partner's; every lane of the warp
// must call it together
template <int D>
__device__ __forceinline__ void gather2(const double* half, int h, double* full) {
#pragma unroll
  for (int j = 0; j < (D + 1) / 2; ++j) {
    const double other = __shfl_xor_sync(0xffffffffu, half[j], 1);
    full[2 * j] = h ? other : half[j];
    if (2 * j + 1 < D) full[2 * j + 1] = h ? half[j] : other;
  }
}

// rows k = 2j + h of L v for L packed lower (entry e at Mp[e * bs]); 0 for k >= D
template <int D>
__device__ __forceinline__ void lower_rows(const double* Mp, size_t bs, int h, const double* v, double* out) {
#pragma unroll
  for (int j = 0; j < (D + 1) / 2; ++j) {
    const int k = 2 * j + h;
    const int row = k < D ? k * (k + 1) / 2 : 0;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m <= 2 * j; ++m) acc += Mp[(size_t)(row + m) * bs] * v[m];
    if (2 * j + 1 < D) {
      const double c = h ? Mp[(size_t)tri(2 * j + 1, 2 * j + 1) * bs] : 0.0;
      acc += c * v[2 * j + 1];
    }
    out[j] = k < D ? acc : 0.0;
  }
}

// rows k = 2j + h of L' v for L packed lower; 0 for k >= D
template <int D>
__device__ __forceinline__ void upper_rows(const double* Mp, size_t bs, int h, const double* v, double* out) {
#pragma unroll
  for (int j = 0; j < (D + 1) / 2; ++j) {
    const int k = 2 * j + h;
    double acc = h ? 0.0 : Mp[(size_t)tri(2 * j, 2 * j) * bs] * v[2 * j];
#pragma unroll
    for (int m = 2 * j + 1; m < D; ++m) acc += Mp[(size_t)(m * (m + 1) / 2 + k) * bs] * v[m];
    out[j] = k < D ? acc : 0.0;
  }
}

// rows k = 2j + h of S v for S packed symmetric; 0 for k >= D
template <int D>
__device__ __forceinline__ void sym_rows(const double* Mp, size_t bs, int h, const double* v, double* out) {
#pragma unroll
  for (int j = 0; j < (D + 1) / 2; ++j) {
    const int k = 2 * j + h;
    const int kk = k < D ? k : 0;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      const int e = kk >= m ? kk * (kk + 1) / 2 + m : m * (m + 1) / 2 + kk;
      acc += Mp[(size_t)e * bs] * v[m];
    }
    out[j] = k < D ? acc : 0.0;
  }
}

}  // namespace

template <int D>
__global__ void __launch_bounds__(RB2_MAX_THREADS, 1) k_pcg_rbp2(PcgArgs a) {
  extern __shared__ double smem[];
  __shared__ Shared sh;
  __shared__ int sh_red[RB2_MAX_THREADS / 2], sh_black[RB2_MAX_THREADS / 2];
  __shared__ int sh_cnt[2 * (RB2_MAX_THREADS / 32)];
  __shared__ double cwd[6];
  __shared__ double s[RES_MAX_D];
  grid_barrier_start(a.bar);
  constexpr int NT = ntri(D), J = (D + 1) / 2;
  const int t = threadIdx.x, h = t & 1, q = t >> 1;
  const int ns = a.pair_slots;   // lane pairs of a CTA: the stride of the shared planes
  if (t == 0) slot_weights(a, cwd);
  if (t < D) s[t] = __ldg(a.scale + t);
  // the CTA's voxels blockIdx.x * res_per + (0 .. res_per - 1), split into a red and a black
  // list (every CTA has at most ns of each colour; the host checked it)
  int nred = 0, nblack = 0;
  {
    const int n0 = blockIdx.x * a.res_per + t;
    const bool mine = t < a.res_per && n0 < a.N;
    const bool blk = mine && a.colour[n0] != 0, rd = mine && !blk;
    const int lane = t & 31, warp = t >> 5, nw = (blockDim.x + 31) >> 5;
    const unsigned mr = __ballot_sync(0xffffffffu, rd), mb = __ballot_sync(0xffffffffu, blk);
    if (lane == 0) {
      sh_cnt[2 * warp] = __popc(mr);
      sh_cnt[2 * warp + 1] = __popc(mb);
    }
    __syncthreads();
    int red_before = 0, black_before = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) {
        red_before += sh_cnt[2 * w];
        black_before += sh_cnt[2 * w + 1];
      }
      nred += sh_cnt[2 * w];
      nblack += sh_cnt[2 * w + 1];
    }
    const unsigned below = (1u << lane) - 1u;
    if (rd && red_before + __popc(mr & below) < ns) sh_red[red_before + __popc(mr & below)] = n0;
    if (blk && black_before + __popc(mb & below) < ns) sh_black[black_before + __popc(mb & below)] = n0;
    __syncthreads();
  }
  const int expect = min(a.res_per, a.N - (int)blockIdx.x * a.res_per);
  if (nred > ns || nblack > ns || 2 * ns > (int)blockDim.x || nred + nblack != expect) {
    // the launcher sized the pairs from the colours; a mismatch stops the solve with an error
    // (the other CTAs leave at their next barrier, which polls the error word)
    if (t == 0) atomicCAS(a.bar.err, 0, ERR_LAYOUT_CODE);
    return;
  }
  const bool hr = q < nred && q < ns, hb = q < nblack && q < ns;   // this pair's red / black voxel
  const int nr = hr ? sh_red[q] : 0, nbv = hb ? sh_black[q] : 0;
  const size_t ld = a.ld;
  double* shR = smem;                 // red slot: Dg_r^-1 (symmetric)
  double* shL = smem + NT * ns;       // black slot: L_b (true diagonal)
  double* shM = smem + 2 * NT * ns;   // black slot: L_b^-1
  double* shH = smem + 3 * NT * ns;   // b^
  double* shP = shH + D * ns;         // p
  double* shS = shP + D * ns;         // s = S^ p
  double* shZ = shS + D * ns;         // z = S^ s
  if (q < ns) {
    // lane 0 of the pair prepares the red slot, lane 1 the black one
    const bool mine = h == 0 ? hr : hb;
    const int nn = h == 0 ? nr : nbv;
    double Lf[NT];
#pragma unroll
    for (int e = 0; e < NT; ++e) Lf[e] = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) Lf[tri(i, i)] = 1.0;
    if (mine) {
#pragma unroll
      for (int e = 0; e < NT; ++e) Lf[e] = __ldg(a.mfac + (size_t)e * ld + nn);
    }
    if (h == 0) {
#pragma unroll
      for (int e = 0; e < NT; ++e) shR[e * ns + q] = Lf[e];
      factor_to_inverse<D, double>(shR + q, ns);
    } else {
#pragma unroll
      for (int e = 0; e < NT; ++e) shM[e * ns + q] = Lf[e];
      double Li[NT];
      lower_inverse<D, double>(shM + q, ns, Li);
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          const int e = tri(i, j);
          shL[e * ns + q] = i == j ? 1.0 / Lf[e] : Lf[e];
          shM[e * ns + q] = Li[e];
        }
    }
  }
  int nbr_r[6], nbr_b[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    nbr_r[d] = (hr && d < a.ndir) ? __ldg(a.nbr + (size_t)d * ld + nr) : -1;
    nbr_b[d] = (hb && d < a.ndir) ? __ldg(a.nbr + (size_t)d * ld + nbv) : -1;
  }
  __syncthreads();
  // component 2j + h exists (only the last one of lane 1 may not, for odd D)
  auto valid = [&](int j) -> bool { return 2 * j + 1 < D || h == 0; };
  auto sidx = [&](int j) -> int { return (2 * j + h) * ns + q; };
  // the black voxel's components; x holds x_b outside the iteration, x^ inside it
  double x[J], r[J], w[J], xr[J];   // xr: the red voxel's components of x (final pass)
#pragma unroll
  for (int j = 0; j < J; ++j) {
    x[j] = (hb && valid(j)) ? a.x[(size_t)(2 * j + h) * ld + nbv] : 0.0;
    r[j] = w[j] = xr[j] = 0.0;
  }
  // lanes past the last pair (padding to whole warps) compute on slot 0 and store nothing
  const int qs = q < ns ? q : 0;
  const double* Rp = shR + qs;
  const double* Lp = shL + qs;
  const double* Mp = shM + qs;
  double* U = a.u;
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  auto scale_of = [&](int j) -> double { return valid(j) ? s[2 * j + h] : 0.0; };
  auto publish = [&](int n, const double* v) {
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (valid(j)) U[(size_t)(2 * j + h) * ld + n] = v[j];
  };
  auto load_b = [&](bool has, int n, double* bv) {
#pragma unroll
    for (int j = 0; j < J; ++j) bv[j] = (has && valid(j)) ? __ldg(a.b + (size_t)(2 * j + h) * ld + n) : 0.0;
  };
  // this lane's components of the weighted neighbour sum of V over the slots nb
  auto nsum = [&](const int* nb, const double* V, double* sum) {
#pragma unroll
    for (int j = 0; j < J; ++j) sum[j] = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (nb[d] >= 0) {
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (valid(j)) sum[j] += cwd[d] * ldx(V + (size_t)(2 * j + h) * ld + nb[d]);
      }
    }
  };
  // the red voxel: out = Dg_r^-1 (c + scale .* sum of the black neighbours' U); every lane
  // calls it
  auto red_solve = [&](const double* c, double* out) {
    double sum[J], tv[J], tf[D];
    nsum(nbr_r, U, sum);
#pragma unroll
    for (int j = 0; j < J; ++j) tv[j] = (c ? c[j] : 0.0) + scale_of(j) * sum[j];
    gather2<D>(tv, h, tf);
    sym_rows<D>(Rp, ns, h, tf, out);
  };
  // this lane's rows of B~ v at voxel n (data block from global memory), V the published v
  // of every voxel; vf the whole v of voxel n, vh this lane's components
  auto amul_rows = [&](int n, const int* nb, const double* vf, const double* vh, const double* V,
                       double* out) {
    double bv[J], sum[J];
    sym_rows<D>(a.blocks + n, ld, h, vf, bv);
    nsum(nb, V, sum);
    const double degd = degree_of<double>(nb, cwd);
#pragma unroll
    for (int j = 0; j < J; ++j) out[j] = valid(j) ? bv[j] + scale_of(j) * (degd * vh[j] - sum[j]) : 0.0;
  };
  // red phase of a product: y = Dg_r^-1 (scale .* sum of the black neighbours' U), published
  auto red_phase = [&]() {
    double y[J];
    red_solve(nullptr, y);
    if (hr) publish(nr, y);
  };
  // out = S^ v at the black voxels (see k_pcg_rbp)
  auto apply_Sh = [&](const double* v, double* out) -> bool {
    double vf[D], vt[J];
    gather2<D>(v, h, vf);
    upper_rows<D>(Mp, ns, h, vf, vt);
    if (hb) publish(nbv, vt);
    if (!bar()) return false;
    red_phase();
    if (!bar()) return false;
    double sum[J], tv[J], tf[D], nn[J];
    nsum(nbr_b, U, sum);
#pragma unroll
    for (int j = 0; j < J; ++j) tv[j] = scale_of(j) * sum[j];
    gather2<D>(tv, h, tf);
    lower_rows<D>(Mp, ns, h, tf, nn);
    if (hb) {
#pragma unroll
      for (int j = 0; j < J; ++j) out[j] = v[j] - nn[j];
    }
    return true;
  };
  // out = S v at the black voxels in unscaled variables (restarts only)
  auto apply_S = [&](const double* v, double* out) -> bool {
    if (hb) publish(nbv, v);
    if (!bar()) return false;
    red_phase();
    if (!bar()) return false;
    double vf[D];
    gather2<D>(v, h, vf);
    if (hb) amul_rows(nbv, nbr_b, vf, v, U, out);
    return true;
  };
  // x_b = L_b^-T x^, then the red voxels from their rows
  auto recover_red = [&]() -> bool {
    double xf[D], xb[J];
    gather2<D>(x, h, xf);
    upper_rows<D>(Mp, ns, h, xf, xb);
    if (hb) {
#pragma unroll
      for (int j = 0; j < J; ++j) x[j] = xb[j];
      publish(nbv, x);
    }
    if (!bar()) return false;
    double bv[J];
    load_b(hr, nr, bv);
    red_solve(bv, xr);
    return true;
  };
  auto true_residual = [&](double* tot) -> bool {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (!valid(j)) continue;
      if (hb) a.x[(size_t)(2 * j + h) * ld + nbv] = x[j];
      if (hr) a.x[(size_t)(2 * j + h) * ld + nr] = xr[j];
    }
    if (!bar()) return false;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    double xf[D], bv[J], ax[J];
    gather2<D>(x, h, xf);
    if (hb) {
      load_b(true, nbv, bv);
      amul_rows(nbv, nbr_b, xf, x, a.x, ax);
#pragma unroll
      for (int j = 0; j < J; ++j) v[2] += (bv[j] - ax[j]) * (bv[j] - ax[j]);
    }
    gather2<D>(xr, h, xf);
    if (hr) {
      load_b(true, nr, bv);
      amul_rows(nr, nbr_r, xf, xr, a.x, ax);
#pragma unroll
      for (int j = 0; j < J; ++j) v[2] += (bv[j] - ax[j]) * (bv[j] - ax[j]);
    }
    return grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };
  // (re)start from the current x_b: r^ = L_b^-1 (b^ - S x_b), x^ = L_b' x_b, w^ = S^ r^,
  // p = s = z = 0
  auto restart = [&]() -> bool {
    double sx[J];
#pragma unroll
    for (int j = 0; j < J; ++j) sx[j] = 0.0;
    if (!apply_S(x, sx)) return false;
    double rb[J], rbf[D], xf[D], rh[J], xh[J];
#pragma unroll
    for (int j = 0; j < J; ++j) rb[j] = (hb && valid(j)) ? shH[sidx(j)] - sx[j] : 0.0;
    gather2<D>(rb, h, rbf);
    gather2<D>(x, h, xf);
    lower_rows<D>(Mp, ns, h, rbf, rh);
    upper_rows<D>(Lp, ns, h, xf, xh);
    if (hb) {
#pragma unroll
      for (int j = 0; j < J; ++j) {
        r[j] = rh[j];
        x[j] = xh[j];
      }
    }
    if (!apply_Sh(r, w)) return false;
    if (hb) {
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (valid(j)) shP[sidx(j)] = shS[sidx(j)] = shZ[sidx(j)] = 0.0;
    }
    return true;
  };

  // b^ = b_b + scale .* sum of the red neighbours' Dg_r^-1 b_r
  {
    double bv[J], bf[D], y[J];
    load_b(hr, nr, bv);
    gather2<D>(bv, h, bf);
    sym_rows<D>(Rp, ns, h, bf, y);
    if (hr) publish(nr, y);
  }
  if (!bar()) return;
  if (hb) {
    double sum[J], bv[J];
    nsum(nbr_b, U, sum);
    load_b(true, nbv, bv);
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (valid(j)) shH[sidx(j)] = bv[j] + s[2 * j + h] * sum[j];
  }
  if (!restart()) return;   // (apply_S's first barrier orders the reads of U above)
  double tot[4];
  double bb = 0.0, tol2 = 0.0, rel0 = 0.0, rr = 0.0;
  double alpha = 0.0, beta = 0.0, gam = 0.0, rgam = 0.0, ralpha = 0.0;
  int it = 0, restarts = 0, status = 0;
  bool first = true;        // first pass of the solve: the partials carry b'b
  bool x_final = false;     // x holds x_b (and the red voxels are recovered)
  while (true) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    {
      // v = L_b^-T w^ first, so that its stores are in flight during the block reduction
      double wf[D], rf[D], vt[J], lr[J];
      gather2<D>(w, h, wf);
      gather2<D>(r, h, rf);
      upper_rows<D>(Mp, ns, h, wf, vt);
      if (hb) publish(nbv, vt);
      lower_rows<D>(Lp, ns, h, rf, lr);
      if (hb) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          v[0] += r[j] * r[j];
          v[1] += w[j] * r[j];
          v[2] += lr[j] * lr[j];
        }
      }
    }
    if (first) {
      double bv[J];
      load_b(hb, nbv, bv);
#pragma unroll
      for (int j = 0; j < J; ++j) v[3] += bv[j] * bv[j];
      load_b(hr, nr, bv);
#pragma unroll
      for (int j = 0; j < J; ++j) v[3] += bv[j] * bv[j];
    }
    const double* part = allreduce4_post(a.part, a.part1, v, sh.red);
    if (!bar()) return;                 // partials and v are visible everywhere
    red_phase();
    allreduce4_collect(part, sh.red, tot, 0);
    if (first) {
      bb = tot[3];
      tol2 = a.delta * a.delta * bb;
      rel0 = bb > 0.0 ? sqrt(tot[2] / bb) : 0.0;
      first = false;
      if (!(isfinite(tot[0]) && isfinite(tot[1]) && isfinite(bb))) status = 7;
    }
    rr = tot[2];
    if (status == 0 && bb == 0.0) {
#pragma unroll
      for (int j = 0; j < J; ++j) x[j] = xr[j] = 0.0;
      x_final = true;
    }
    int code = 0;
    if (status == 0 && bb != 0.0) {
      cg_scalar_step(sh, tot[0], tot[1], rr, tol2, it, a.max_iter, alpha, beta, gam, rgam, ralpha);
      code = sh.code;
      __syncthreads();
    }
    if (!bar()) return;                 // the red phase's y is visible; all partials read
    if (status != 0 || bb == 0.0) break;
    if (code == 7) { status = 7; break; }
    if (code == 3) { status = 3; break; }
    if (code == 1) {
      // confirm with the true residual of B~
      if (!recover_red()) return;
      if (!true_residual(tot)) return;
      x_final = true;
      rr = tot[2];
      if (rr <= tol2) break;
      if (it >= a.max_iter) { status = 4; break; }
      ++restarts;
      if (!restart()) return;
      x_final = false;
      rgam = 0.0;
      ralpha = 0.0;
      continue;
    }
    {
      double sum[J], tv[J], tf[D], nn[J];
      nsum(nbr_b, U, sum);
#pragma unroll
      for (int j = 0; j < J; ++j) tv[j] = scale_of(j) * sum[j];
      gather2<D>(tv, h, tf);
      lower_rows<D>(Mp, ns, h, tf, nn);   // n = w^ - L_b^-1 (scale .* sum y)
      if (hb) {
        const double al = alpha, be = beta;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          if (!valid(j)) continue;
          const int o = sidx(j);
          const double z = (w[j] - nn[j]) + be * shZ[o];
          const double sv = w[j] + be * shS[o];
          const double p = r[j] + be * shP[o];
          shZ[o] = z;
          shS[o] = sv;
          shP[o] = p;
          x[j] += al * p;
          r[j] -= al * sv;
          w[j] -= al * z;
        }
      }
    }
    ++it;
  }
  if (!x_final && !recover_red()) return;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    if (!valid(j)) continue;
    if (hb) a.x[(size_t)(2 * j + h) * ld + nbv] = x[j];
    if (hr) a.x[(size_t)(2 * j + h) * ld + nr] = xr[j];
  }
  write_ctrl(a, it, restarts, rr, bb, rel0, status);
}

// ---------------------------------------------------------------------------------------
// Mixed precision on the red-black reduced system (resident): FP64 iterative refinement of
// the full system (true residual r of B~ over every voxel, x += d), each correction d from
// FP32 pipelined CG on the reduced system of B~ d = r,
//   S d_b = r_b + scale .* sum_red nbrs Dg_r^-1 r_r,  d_r = Dg_r^-1 (r_r + scale .* sum d_b),
// with float-float partial sums posted before the product's first barrier and collected
// after it (two barriers per inner iteration, as k_pcg_rbp) and explicit FP32 block inverses.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(RES_MAX_THREADS, 1) k_pcg_mixed_rbp(PcgArgs a) {
  extern __shared__ double smem[];
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  __shared__ double cwd[6];
  __shared__ float cwf[6];
  if (threadIdx.x == 0) {
    slot_weights(a, cwd);
    slot_weights(a, cwf);
  }
  __syncthreads();
  constexpr int NT = ntri(D);
  const int bd = blockDim.x, t = threadIdx.x;
  double* shB = smem;                                   // [NT][bd] FP64 blocks
  float* shB32 = reinterpret_cast<float*>(smem + NT * bd);   // [NT][bd]
  float* shM32 = shB32 + NT * bd;                       // [NT][bd] block inverses (FP32)
  int n = blockIdx.x * a.res_per + t;
  bool own = t < a.res_per && n < a.N;
  bool is_red = true;
  colour_sort(a, n, own, is_red);
  const bool red = own && is_red, black = own && !is_red;
  const size_t ld = a.ld;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const int e = tri(i, j);
      shB[e * bd + t] = own ? __ldg(a.blocks + (size_t)e * ld + n) : (i == j ? 1.0 : 0.0);
      shB32[e * bd + t] = own ? __ldg(a.blocks32 + (size_t)e * ld + n) : (i == j ? 1.f : 0.f);
      shM32[e * bd + t] = own ? __ldg(a.mfac32 + (size_t)e * ld + n) : (i == j ? 1.f : 0.f);
    }
  factor_to_inverse<D, float>(shM32 + t, bd);
  int nb[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) nb[d] = (own && d < a.ndir) ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  const double degd = degree_of<double>(nb, cwd);
  const float degf = (float)degd;
  double s[D], x[D], bv[D];
  float s32[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    s[k] = __ldg(a.scale + k);
    s32[k] = (float)s[k];
    x[k] = own ? a.x[(size_t)k * ld + n] : 0.0;
    bv[k] = own ? __ldg(a.b + (size_t)k * ld + n) : 0.0;
  }
  const double* Bp = shB + t;
  const float* Bp32 = shB32 + t;
  const float* Mp32 = shM32 + t;
  float* U = a.u32;
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  auto publish = [&](const float* v) {
#pragma unroll
    for (int k = 0; k < D; ++k) U[(size_t)k * ld + n] = v[k];
  };
  auto red_solve = [&](const float* c, float* out) {
    float sum[D], tv[D];
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] = 0.f;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (nb[d] >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += cwf[d] * ldx(U + (size_t)k * ld + nb[d]);
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) tv[k] = (c ? c[k] : 0.f) + s32[k] * sum[k];
    symv<D, float>(Mp32, bd, tv, out);
  };
  auto apply_S = [&](const float* v, float* out) -> bool {
    if (black) publish(v);
    if (!bar()) return false;
    if (red) {
      float y[D];
      red_solve(nullptr, y);
      publish(y);
    }
    if (!bar()) return false;
    if (black) amul<D, float>(Bp32, bd, s32, nb, cwf, degf, v, U, ld, out);
    return true;
  };
  double tot[4];
  int outer = 0, inner_total = 0, status = 0;
  double bb = 0.0, rr = 0.0, rel0 = 0.0, tol2 = 0.0;
  while (true) {
    // ---- FP64 true residual (x of every voxel is complete: start value or published) ----
    double r64[D];
    {
      double ax[D];
      amul<D, double>(Bp, bd, s, nb, cwd, degd, x, a.x, ld, ax);
      double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < D; ++k) {
        r64[k] = bv[k] - ax[k];
        v[0] += r64[k] * r64[k];
        v[1] += bv[k] * bv[k];
      }
      if (!grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    }
    rr = tot[0];
    if (outer == 0) {
      bb = tot[1];
      tol2 = a.delta * a.delta * bb;
      rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      if (!(isfinite(rr) && isfinite(bb))) { status = 7; break; }
      if (bb == 0.0) {
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = 0.0;
        break;
      }
    }
    if (!isfinite(rr)) { status = 7; break; }
    if (rr <= tol2) break;
    if (inner_total >= a.max_iter) { status = 4; break; }
    ++outer;
    // ---- FP32 pipelined CG on the reduced system of B~ d = r ----
    float rc[D], r[D], u[D], w[D], d[D], p[D], sv[D], q[D], z[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      rc[k] = (float)r64[k];
      r[k] = u[k] = w[k] = d[k] = p[k] = sv[k] = q[k] = z[k] = 0.f;
    }
    const double itol2 = fmax(a.inner_tol * a.inner_tol * rr, 0.25 * tol2);
    if (red) {
      float y[D];
      symv<D, float>(Mp32, bd, rc, y);
      publish(y);
    }
    if (!bar()) return;
    if (black) {
      float sum[D];
#pragma unroll
      for (int k = 0; k < D; ++k) sum[k] = 0.f;
#pragma unroll
      for (int dd = 0; dd < 6; ++dd) {
        if (nb[dd] >= 0) {
#pragma unroll
          for (int k = 0; k < D; ++k) sum[k] += cwf[dd] * ldx(U + (size_t)k * ld + nb[dd]);
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) r[k] = rc[k] + s32[k] * sum[k];
      symv<D, float>(Mp32, bd, r, u);
    }
    if (!apply_S(u, w)) return;   // its first barrier orders the reads of U above
    double alpha = 0.0, beta = 0.0, gam = 0.0, rgam = 0.0, ralpha = 0.0;
    int it = 0;
    while (true) {
      float g = 0.f, dl = 0.f, q2 = 0.f;
      if (black) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          g += r[k] * u[k];
          dl += w[k] * u[k];
          q2 += r[k] * r[k];
        }
      }
      // m = M^-1 w published before the block reduction, so that its stores are in flight
      float m[D];
      if (black) {
        symv<D, float>(Mp32, bd, w, m);
        publish(m);
      }
      const FF v[4] = {ff_of(g), ff_of(dl), ff_of(q2), ff_of(0.f)};
      const float* part = allreduce4_ff_post(a.part, a.part1, v, sh.red);
      if (!bar()) return;                 // partials and m are visible everywhere
      if (red) {
        float y[D];
        red_solve(nullptr, y);
        publish(y);
      }
      // the loads run on the last four warps (black voxels or none, idle in the red phase)
      allreduce4_ff_collect(part, sh.red, tot, bd >= 128 ? (bd >> 5) - 4 : 0);
      const bool capped = it >= a.max_inner || inner_total + it >= a.max_iter;
      cg_scalar_step(sh, tot[0], tot[1], tot[2], itol2, capped ? 1 : 0, 1, alpha, beta, gam, rgam, ralpha);
      const int code = sh.code;
      __syncthreads();
      if (!bar()) return;                 // y visible; every CTA has read the partials
      if (code == 7) { status = 7; break; }
      if (code != 0) break;   // inner tolerance, iteration cap, or loss of conjugacy in FP32
      if (black) {
        float nn[D];
        amul<D, float>(Bp32, bd, s32, nb, cwf, degf, m, U, ld, nn);   // n = S m
        const float fa = (float)alpha, fb = (float)beta;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          z[k] = nn[k] + fb * z[k];
          q[k] = m[k] + fb * q[k];
          sv[k] = w[k] + fb * sv[k];
          p[k] = u[k] + fb * p[k];
          d[k] += fa * p[k];
          r[k] -= fa * sv[k];
          u[k] -= fa * q[k];
          w[k] -= fa * z[k];
        }
      }
      ++it;
    }
    inner_total += it;
    if (status != 0) break;
    // red part of the correction from the red rows, then x += d everywhere
    if (black) publish(d);
    if (!bar()) return;
    if (red) red_solve(rc, d);
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] += (double)d[k];
    if (own) {
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
    }
    if (!bar()) return;
  }
  if (own) {
#pragma unroll
    for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = x[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->iterations = inner_total;
    a.ctrl->restarts = outer;
    a.ctrl->rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    a.ctrl->rel_res0 = rel0;
    a.ctrl->status = status;
    if (status != 0 && a.ctrl->status_any == 0) a.ctrl->status_any = status;
    a.ctrl->iter_total += inner_total;
    a.ctrl->solves += 1;
  }
}


// ---------------------------------------------------------------------------------------
// Mixed precision (streaming): the same refinement with vectors in global memory.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_mixed_stream(PcgArgs a) {
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  // per-slot edge weights in shared memory (read as broadcasts; no registers held)
  __shared__ double cwd[6];
  __shared__ float cwf[6];
  if (threadIdx.x == 0) {
    slot_weights(a, cwd);
    slot_weights(a, cwf);
  }
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const size_t ld = a.ld;
  const bool pre = a.mfac32 != nullptr;
  double s[D];
  float s32[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    s[k] = __ldg(a.scale + k);
    s32[k] = (float)s[k];
  }
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  auto load_nb = [&](int n, int* nb) {
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = d < a.ndir ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  };
  auto precond = [&](int n, const float* rn, float* un) {
    if (pre) {
      minv<D, float>(a.mfac32 + n, (int)ld, rn, un);
      if (a.ssor) {
#pragma unroll
        for (int k = 0; k < D; ++k) un[k] *= (float)a.omega;   // SSOR phase 1
      }
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) un[k] = rn[k];
    }
  };
  // SSOR phases 2 (black voxels) and 3 (red voxels) of the inner iterations, each after a barrier
  auto ssor_rest = [&]() -> bool {
    if (!bar()) return false;
    for (int i = tid; i < a.n_black; i += nth) ssor_phase<D, float>(a, s32, a.mfac32, a.r32, a.u32, a.black[i], 2);
    if (!bar()) return false;
    for (int i = tid; i < a.n_red; i += nth) ssor_phase<D, float>(a, s32, a.mfac32, a.r32, a.u32, a.red[i], 3);
    return true;
  };
  // inner matvec phase: w = B~ u and the three partial sums
  auto matvec_partials = [&](double* tot) -> bool {
    FF v[4] = {ff_of(0.f), ff_of(0.f), ff_of(0.f), ff_of(0.f)};
    for (int n = tid; n < a.N; n += nth) {
      int nb[6];
      load_nb(n, nb);
      float un[D], wn[D], rk[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        un[k] = a.u32[(size_t)k * ld + n];
        rk[k] = a.r32[(size_t)k * ld + n];
      }
      amul<D, float>(a.blocks32 + n, (int)ld, s32, nb, cwf, degree_of<float>(nb, cwf), un, a.u32, ld, wn);
      float g = 0.f, dl = 0.f, q2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        g += rk[k] * un[k];
        dl += wn[k] * un[k];
        q2 += rk[k] * rk[k];
      }
#pragma unroll
      for (int k = 0; k < D; ++k) a.w32[(size_t)k * ld + n] = wn[k];
      v[0] = ff_add(v[0], ff_of(g));
      v[1] = ff_add(v[1], ff_of(dl));
      v[2] = ff_add(v[2], ff_of(q2));
    }
    return grid_allreduce4_ff(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };
  double tot[4];
  int outer = 0, inner_total = 0, status = 0;
  double bb = 0.0, rr = 0.0, rel0 = 0.0, tol2 = 0.0;
  while (true) {
    {
      double v[4] = {0.0, 0.0, 0.0, 0.0};
      for (int n = tid; n < a.N; n += nth) {
        int nb[6];
        load_nb(n, nb);
        double xn[D], ax[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xn[k] = ldx(a.x + (size_t)k * ld + n);
        amul<D, double>(a.blocks + n, (int)ld, s, nb, cwd, degree_of<double>(nb, cwd), xn, a.x, ld, ax);
        float rn[D], un[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double bk = __ldg(a.b + (size_t)k * ld + n);
          const double rk = bk - ax[k];
          v[0] += rk * rk;
          v[1] += bk * bk;
          rn[k] = (float)rk;
        }
        precond(n, rn, un);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          a.r32[(size_t)k * ld + n] = rn[k];
          a.u32[(size_t)k * ld + n] = un[k];
          a.d32[(size_t)k * ld + n] = 0.f;
          a.p32[(size_t)k * ld + n] = 0.f;
          a.s32[(size_t)k * ld + n] = 0.f;
        }
      }
      if (!grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    }
    rr = tot[0];
    if (outer == 0) {
      bb = tot[1];
      tol2 = a.delta * a.delta * bb;
      rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      if (!(isfinite(rr) && isfinite(bb))) { status = 7; break; }
      if (bb == 0.0) {
        for (int n = tid; n < a.N; n += nth)
#pragma unroll
          for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = 0.0;
        break;
      }
    }
    if (!isfinite(rr)) { status = 7; break; }
    if (rr <= tol2) break;
    if (inner_total >= a.max_iter) { status = 4; break; }
    ++outer;
    // inner target: inner_tol relative, but no further than the outer stop needs
    const double itol2 = fmax(a.inner_tol * a.inner_tol * rr, 0.25 * tol2);
    // u was published by the residual phase, whose reducing barrier has completed
    if (a.ssor && (!ssor_rest() || !bar())) return;
    if (!matvec_partials(tot)) return;
    double gam = tot[0], del = tot[1];
    if (!(del > 0.0) || !isfinite(del)) { status = isfinite(del) ? 3 : 7; break; }
    double alpha = gam / del, beta = 0.0;
    double rgam = 0.0, ralpha = 0.0;
    cg_recips(gam, del, rgam, ralpha);
    int it = 0;
    while (true) {
      const float fa = (float)alpha, fb = (float)beta;
      for (int n = tid; n < a.N; n += nth) {
        float rn[D], un[D], pk[D], sk[D], dk[D], wk[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const size_t o = (size_t)k * ld + n;
          un[k] = a.u32[o];
          pk[k] = a.p32[o];
          wk[k] = a.w32[o];
          sk[k] = a.s32[o];
          dk[k] = a.d32[o];
          rn[k] = a.r32[o];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          pk[k] = un[k] + fb * pk[k];
          sk[k] = wk[k] + fb * sk[k];
          dk[k] += fa * pk[k];
          rn[k] -= fa * sk[k];
        }
        precond(n, rn, un);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const size_t o = (size_t)k * ld + n;
          a.p32[o] = pk[k];
          a.s32[o] = sk[k];
          a.d32[o] = dk[k];
          a.r32[o] = rn[k];
          a.u32[o] = un[k];
        }
      }
      if (a.ssor && !ssor_rest()) return;
      if (!bar()) return;
      if (!matvec_partials(tot)) return;
      ++it;
      const bool capped = it >= a.max_inner || inner_total + it >= a.max_iter;
      cg_scalar_step(sh, tot[0], tot[1], tot[2], itol2, capped ? 1 : 0, 1, alpha, beta, gam, rgam, ralpha);
      const int code = sh.code;
      __syncthreads();
      if (code == 7) { status = 7; break; }
      if (code != 0) break;   // inner tolerance, iteration cap, or loss of conjugacy in FP32
    }
    inner_total += it;
    if (status != 0) break;
    for (int n = tid; n < a.N; n += nth)
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] += (double)a.d32[(size_t)k * ld + n];
    if (!bar()) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->iterations = inner_total;
    a.ctrl->restarts = outer;
    a.ctrl->rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    a.ctrl->rel_res0 = rel0;
    a.ctrl->status = status;
    if (status != 0 && a.ctrl->status_any == 0) a.ctrl->status_any = status;
    a.ctrl->iter_total += inner_total;
    a.ctrl->solves += 1;
  }
}

// ---------------------------------------------------------------------------------------
// Streaming mixed precision on the red-black reduced system (any N): the FP64 refinement of
// k_pcg_mixed_stream, each correction from FP32 CG on the reduced system of B~ d = r with
// the vectors in global memory. Black voxels run over the black list, red ones over the red
// list. r32 holds r~ at the black voxels and the red part of the refinement right-hand side
// at the red ones; u32 carries u at the black voxels and y = Dg_r^-1 (...) at the red ones;
// d32 holds the correction at both.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg_mixed_stream_rb(PcgArgs a) {
  __shared__ Shared sh;
  grid_barrier_start(a.bar);
  __shared__ double cwd[6];
  __shared__ float cwf[6];
  if (threadIdx.x == 0) {
    slot_weights(a, cwd);
    slot_weights(a, cwf);
  }
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const size_t ld = a.ld;
  double s[D];
  float s32[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    s[k] = __ldg(a.scale + k);
    s32[k] = (float)s[k];
  }
  auto bar = [&]() -> bool {
    if (a.skip_block == (int)blockIdx.x) return false;
    return grid_sync(a.bar, &sh.flag);
  };
  auto load_nb = [&](int n, int* nb) {
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = d < a.ndir ? __ldg(a.nbr + (size_t)d * ld + n) : -1;
  };
  // out = Dg_n^-1 (c + scale .* sum of the neighbours' V), FP32
  auto colour_solve = [&](int n, const float* c, const float* V, float* out) {
    int nb[6];
    load_nb(n, nb);
    float sum[D], tv[D];
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] = 0.f;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      if (nb[d] >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += cwf[d] * ldx(V + (size_t)k * ld + nb[d]);
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) tv[k] = (c ? c[k] : 0.f) + s32[k] * sum[k];
    minv<D, float>(a.mfac32 + n, (int)ld, tv, out);
  };
  auto store = [&](float* V, int n, const float* v) {
#pragma unroll
    for (int k = 0; k < D; ++k) V[(size_t)k * ld + n] = v[k];
  };
  auto load = [&](const float* V, int n, float* v) {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = V[(size_t)k * ld + n];
  };
  // red phase (u32 at the red voxels from u at the black ones), barrier, black product
  // w = S u with the partials (r'u, w'u, r'r)
  auto product_partials = [&](double* tot) -> bool {
    for (int i = tid; i < a.n_red; i += nth) {
      const int n = __ldg(a.red + i);
      float y[D];
      colour_solve(n, nullptr, a.u32, y);
      store(a.u32, n, y);
    }
    if (!bar()) return false;
    FF v[4] = {ff_of(0.f), ff_of(0.f), ff_of(0.f), ff_of(0.f)};
    for (int i = tid; i < a.n_black; i += nth) {
      const int n = __ldg(a.black + i);
      int nb[6];
      load_nb(n, nb);
      float un[D], wn[D], rk[D];
      load(a.u32, n, un);
      load(a.r32, n, rk);
      amul<D, float>(a.blocks32 + n, (int)ld, s32, nb, cwf, degree_of<float>(nb, cwf), un, a.u32, ld, wn);
      float g = 0.f, dl = 0.f, q2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        g += rk[k] * un[k];
        dl += wn[k] * un[k];
        q2 += rk[k] * rk[k];
      }
      store(a.w32, n, wn);
      v[0] = ff_add(v[0], ff_of(g));
      v[1] = ff_add(v[1], ff_of(dl));
      v[2] = ff_add(v[2], ff_of(q2));
    }
    return grid_allreduce4_ff(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot);
  };
  double tot[4];
  int outer = 0, inner_total = 0, status = 0;
  double bb = 0.0, rr = 0.0, rel0 = 0.0, tol2 = 0.0;
  while (true) {
    // ---- FP64 true residual over every voxel; its FP32 copy goes to r32 ----
    {
      double v[4] = {0.0, 0.0, 0.0, 0.0};
      for (int n = tid; n < a.N; n += nth) {
        int nb[6];
        load_nb(n, nb);
        double xn[D], ax[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xn[k] = ldx(a.x + (size_t)k * ld + n);
        amul<D, double>(a.blocks + n, (int)ld, s, nb, cwd, degree_of<double>(nb, cwd), xn, a.x, ld, ax);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double bk = __ldg(a.b + (size_t)k * ld + n);
          const double rk = bk - ax[k];
          v[0] += rk * rk;
          v[1] += bk * bk;
          a.r32[(size_t)k * ld + n] = (float)rk;
          a.d32[(size_t)k * ld + n] = 0.f;
        }
      }
      if (!grid_allreduce4(a.bar, a.part, a.part1, v, sh.red, sh.ints, tot)) return;
    }
    rr = tot[0];
    if (outer == 0) {
      bb = tot[1];
      tol2 = a.delta * a.delta * bb;
      rel0 = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      if (!(isfinite(rr) && isfinite(bb))) { status = 7; break; }
      if (bb == 0.0) {
        for (int n = tid; n < a.N; n += nth)
#pragma unroll
          for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] = 0.0;
        break;
      }
    }
    if (!isfinite(rr)) { status = 7; break; }
    if (rr <= tol2) break;
    if (inner_total >= a.max_iter) { status = 4; break; }
    ++outer;
    const double itol2 = fmax(a.inner_tol * a.inner_tol * rr, 0.25 * tol2);
    // reduced right-hand side: y0 = Dg_r^-1 r_r at the red voxels, then at the black ones
    // r~ = r_b + scale .* sum y0, u = Dg_b^-1 r~, p = s = 0
    for (int i = tid; i < a.n_red; i += nth) {
      const int n = __ldg(a.red + i);
      float rc[D], y[D];
      load(a.r32, n, rc);
      minv<D, float>(a.mfac32 + n, (int)ld, rc, y);
      store(a.u32, n, y);
    }
    if (!bar()) return;
    // (black voxels write u32 only at black voxels and read it only at red ones)
    for (int i = tid; i < a.n_black; i += nth) {
      const int n = __ldg(a.black + i);
      float rc[D], rt[D], un[D], zero[D];
      load(a.r32, n, rc);
      int nb[6];
      load_nb(n, nb);
      float sum[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        sum[k] = 0.f;
        zero[k] = 0.f;
      }
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        if (nb[d] >= 0) {
#pragma unroll
          for (int k = 0; k < D; ++k) sum[k] += cwf[d] * ldx(a.u32 + (size_t)k * ld + nb[d]);
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) rt[k] = rc[k] + s32[k] * sum[k];
      minv<D, float>(a.mfac32 + n, (int)ld, rt, un);
      store(a.r32, n, rt);
      store(a.u32, n, un);
      store(a.p32, n, zero);
      store(a.s32, n, zero);
    }
    if (!bar()) return;
    if (!product_partials(tot)) return;
    double gam = tot[0], del = tot[1];
    if (!(del > 0.0) || !isfinite(del)) { status = isfinite(del) ? 3 : 7; break; }
    double alpha = gam / del, beta = 0.0;
    double rgam = 0.0, ralpha = 0.0;
    cg_recips(gam, del, rgam, ralpha);
    int it = 0;
    while (true) {
      const float fa = (float)alpha, fb = (float)beta;
      for (int i = tid; i < a.n_black; i += nth) {
        const int n = __ldg(a.black + i);
        float rn[D], un[D], pk[D], sk[D], dk[D], wk[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const size_t o = (size_t)k * ld + n;
          un[k] = a.u32[o];
          pk[k] = a.p32[o];
          wk[k] = a.w32[o];
          sk[k] = a.s32[o];
          dk[k] = a.d32[o];
          rn[k] = a.r32[o];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          pk[k] = un[k] + fb * pk[k];
          sk[k] = wk[k] + fb * sk[k];
          dk[k] += fa * pk[k];
          rn[k] -= fa * sk[k];
        }
        minv<D, float>(a.mfac32 + n, (int)ld, rn, un);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const size_t o = (size_t)k * ld + n;
          a.p32[o] = pk[k];
          a.s32[o] = sk[k];
          a.d32[o] = dk[k];
          a.r32[o] = rn[k];
          a.u32[o] = un[k];
        }
      }
      if (!bar()) return;
      if (!product_partials(tot)) return;
      ++it;
      const bool capped = it >= a.max_inner || inner_total + it >= a.max_iter;
      cg_scalar_step(sh, tot[0], tot[1], tot[2], itol2, capped ? 1 : 0, 1, alpha, beta, gam, rgam, ralpha);
      const int code = sh.code;
      __syncthreads();
      if (code == 7) { status = 7; break; }
      if (code != 0) break;   // inner tolerance, iteration cap, or loss of conjugacy in FP32
    }
    inner_total += it;
    if (status != 0) break;
    // red part of the correction from the red rows (d32 at the black voxels is final), then
    // x += d everywhere
    for (int i = tid; i < a.n_red; i += nth) {
      const int n = __ldg(a.red + i);
      float rc[D], dn[D];
      load(a.r32, n, rc);
      colour_solve(n, rc, a.d32, dn);
      store(a.d32, n, dn);
    }
    if (!bar()) return;
    for (int n = tid; n < a.N; n += nth)
#pragma unroll
      for (int k = 0; k < D; ++k) a.x[(size_t)k * ld + n] += (double)a.d32[(size_t)k * ld + n];
    if (!bar()) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->iterations = inner_total;
    a.ctrl->restarts = outer;
    a.ctrl->rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    a.ctrl->rel_res0 = rel0;
    a.ctrl->status = status;
    if (status != 0 && a.ctrl->status_any == 0) a.ctrl->status_any = status;
    a.ctrl->iter_total += inner_total;
    a.ctrl->solves += 1;
  }
}

// ---------------------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------------------
namespace {

inline int num_sms() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

inline int capped_sms(int cap) {
  const int n = num_sms();
  return (cap > 0 && cap < n) ? cap : n;
}

}  // namespace


namespace {

template <int D>
cudaError_t launch_resident(const PcgArgs& a, cudaStream_t stream, int* grid_out, bool* launched) {
  *launched = false;
  const int nsm = capped_sms(a.sm_cap);
  // spread the voxels evenly over the SMs: CTA b owns voxels [b per, (b + 1) per)
  const int per = resident_voxels_per_cta(a.N, a.sm_cap);
  const int grid = (a.N + per - 1) / per;
  int threads = ((per + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  if (threads > (a.reduced && !a.mixed ? RB_MAX_THREADS : RES_MAX_THREADS)) return cudaSuccess;
  if (a.max_grid > 0 && grid > a.max_grid) return cudaSuccess;
  // FP64: blocks + factor in FP64; mixed: FP64 blocks + FP32 blocks + FP32 factor
  // the pipelined reduced solver keeps b^, p, s, z in shared memory: D <= 6
  constexpr bool kPipe = D <= 6;
  // lane pairs (k_pcg_rbp2): one red and one black voxel per pair of lanes; the host sized
  // the pairs for this voxels-per-CTA count
  const bool pair = kPipe && a.reduced && !a.mixed && a.lanes != 1 && a.pair_slots > 0 &&
                    a.pair_per == per && 2 * a.pair_slots <= RB2_MAX_THREADS && !a.scale3 && !a.ce;
  // the anisotropic prior's reduced system: the pipelined one-lane kernel (D <= 6) only
  if (a.scale3 && a.reduced && !kPipe) return cudaSuccess;
  if (pair) threads = std::max(64, ((2 * a.pair_slots + 31) / 32) * 32);
  // per-edge factors: the one-lane FP64 kernels keep six slot weights a voxel after the rest
  const int prior = a.scale3 ? PRIOR_SCALE3 : a.ce ? PRIOR_EDGE : a.ltl ? PRIOR_LTL : PRIOR_DIR;
  if (a.ltl && (a.mixed || a.reduced || a.ssor || a.t == nullptr)) return cudaSuccess;
  if (a.ce && (a.mixed || (a.reduced && !kPipe))) return cudaSuccess;
  const size_t shm = a.mixed ? (size_t)ntri(D) * threads * (sizeof(double) + 2 * sizeof(float))
                     : pair  ? (size_t)(3 * ntri(D) + 4 * D) * a.pair_slots * sizeof(double)
                     : a.reduced ? (size_t)(2 * ntri(D) + (kPipe ? 4 : 1) * D + (a.ce ? 6 : 0)) * threads * sizeof(double)
                                 : (size_t)(2 * ntri(D) + (a.ce ? 6 : 0)) * threads * sizeof(double);
  const void* kred = nullptr;
  if constexpr (kPipe)
    kred = pair ? (const void*)k_pcg_rbp2<D>
                : prior == PRIOR_SCALE3 ? (const void*)k_pcg_rbp<D, PRIOR_SCALE3>
                : prior == PRIOR_EDGE   ? (const void*)k_pcg_rbp<D, PRIOR_EDGE>
                                        : (const void*)k_pcg_rbp<D, PRIOR_DIR>;
  else kred = (const void*)k_pcg_rb<D>;
  const void* kern = a.mixed ? (a.reduced ? (const void*)k_pcg_mixed_rbp<D> : (const void*)k_pcg_mixed_res<D>)
                             : (a.reduced ? kred
                                : prior == PRIOR_SCALE3 ? (const void*)k_pcg_res<D, PRIOR_SCALE3>
                                : prior == PRIOR_EDGE   ? (const void*)k_pcg_res<D, PRIOR_EDGE>
                                : prior == PRIOR_LTL    ? (const void*)k_pcg_res<D, PRIOR_LTL>
                                                        : (const void*)k_pcg_res<D, PRIOR_DIR>);
  if (raise_smem_limit(kern, shm) != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, shm) != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  if (per_sm < 1 || grid > per_sm * nsm) return cudaSuccess;
  if (grid_out) *grid_out = grid;
  *launched = true;
  PcgArgs b = a;
  b.res_per = per;
  cudaError_t er = reset_grid_barrier(b.bar, stream);
  if (er != cudaSuccess) return er;
  void* args[] = {(void*)&b};
  return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, shm, stream);
}

}  // namespace

namespace pcg_detail {

template <int D>
cudaError_t launch_d(const PcgArgs& a, cudaStream_t stream, int* grid_out) {
  if constexpr (D <= RES_MAX_D) {
    // the anisotropic prior and per-edge factors: the block-Jacobi or the reduced resident kernel
    // the L'L prior: the block-Jacobi resident kernel
    if (a.allow_resident && (!a.ltl || (!a.mixed && !a.reduced && !a.ssor)) &&
        (!(a.scale3 || a.ce) || (!a.mixed && (a.reduced || !a.ssor)))) {
      bool launched = false;
      cudaError_t e = launch_resident<D>(a, stream, grid_out, &launched);
      if (launched || e != cudaSuccess) return e;
    }
  }
  const int nsm = capped_sms(a.sm_cap);
  if (a.ltl && (a.mixed || a.ssor || a.reduced || a.t == nullptr)) return cudaErrorInvalidValue;
  if (a.ce && (a.mixed || a.ltl || a.scale3)) return cudaErrorInvalidValue;
  if (a.scale3 && (a.mixed || a.ltl || D > DMAX)) return cudaErrorInvalidValue;
  if ((a.scale3 || a.ce) && (a.ssor || a.reduced)) {
    // the reduced system did not fit the resident kernel: the streaming solver with the same
    // block-Jacobi factor (the reduced system's diagonal blocks) instead of SSOR
    if (a.ssor && !a.reduced) return cudaErrorInvalidValue;
    PcgArgs b = a;
    b.reduced = 0;
    b.ssor = 0;
    return launch_d<D>(b, stream, grid_out);
  }
  const void* kern = a.ltl ? (const void*)k_pcg_ltl<D>
                     : a.mixed ? (a.reduced ? (const void*)k_pcg_mixed_stream_rb<D> : (const void*)k_pcg_mixed_stream<D>)
                               : (const void*)k_pcg_stream<D>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PCG_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int need = (a.N + PCG_THREADS - 1) / PCG_THREADS;
  int grid = nsm * per_sm;
  if (need < grid) grid = need < 1 ? 1 : need;
  if (a.max_grid > 0 && grid > a.max_grid) grid = a.max_grid;
  if (grid_out) *grid_out = grid;
  e = reset_grid_barrier(a.bar, stream);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(PCG_THREADS), args, 0, stream);
}

template <int D>
int max_grid_d() {
  int p1 = 0, p2 = 0, p3 = 0, p4 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_pcg_stream<D>, PCG_THREADS, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_pcg_mixed_stream<D>, PCG_THREADS, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p3, k_pcg_mixed_stream_rb<D>, PCG_THREADS, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, k_pcg_ltl<D>, PCG_THREADS, 0);
  int per_sm = p1 > p2 ? p1 : p2;
  per_sm = per_sm > p3 ? per_sm : p3;
  per_sm = per_sm > p4 ? per_sm : p4;
  return num_sms() * (per_sm > 1 ? per_sm : 1);
}


// Preconditioner inspection: phase 0 = block-Jacobi (or identity), 1..3 = SSOR phases.
template <int D>
__global__ void __launch_bounds__(PCG_THREADS) k_precond_phase(PcgArgs a, int phase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s[D];
#pragma unroll
  for (int k = 0; k < D; ++k) s[k] = __ldg(a.scale + k);
  if (phase <= 1) {
    if (i >= a.N) return;
    double r[D], z[D];
#pragma unroll
    for (int k = 0; k < D; ++k) r[k] = a.r[(size_t)k * a.ld + i];
    if (a.mfac != nullptr) {
      minv<D, double>(a.mfac + i, (int)a.ld, r, z);
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) z[k] = r[k];
    }
    const double f = phase == 1 ? a.omega : 1.0;
#pragma unroll
    for (int k = 0; k < D; ++k) a.u[(size_t)k * a.ld + i] = f * z[k];
  } else if (phase == 2) {
    if (i < a.n_black) ssor_phase<D, double>(a, s, a.mfac, a.r, a.u, a.black[i], 2);
  } else {
    if (i < a.n_red) ssor_phase<D, double>(a, s, a.mfac, a.r, a.u, a.red[i], 3);
  }
}

template <int D>
cudaError_t precond_apply_d(const PcgArgs& a, cudaStream_t stream) {
  const int g = (a.N + PCG_THREADS - 1) / PCG_THREADS;
  if (!a.ssor) {
    k_precond_phase<D><<<g, PCG_THREADS, 0, stream>>>(a, 0);
    return cudaGetLastError();
  }
  if (a.mfac == nullptr) return cudaErrorInvalidValue;
  for (int phase = 1; phase <= 3; ++phase) {
    k_precond_phase<D><<<g, PCG_THREADS, 0, stream>>>(a, phase);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pcg_detail

// explicit instantiation of the three launchers for one D (kernels_pcg_d*.cu)
#define BFMRI_PCG_INSTANTIATE(d)                                                           \
  template cudaError_t pcg_detail::launch_d<d>(const PcgArgs&, cudaStream_t, int*);       \
  template int pcg_detail::max_grid_d<d>();                                                \
  template cudaError_t pcg_detail::precond_apply_d<d>(const PcgArgs&, cudaStream_t);

}  // namespace bfmri
