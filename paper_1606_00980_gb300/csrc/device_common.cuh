// Device helpers shared by the bfmri kernels: counter-based random numbers, packed symmetric
// K x K blocks, a bounded grid barrier and deterministic grid reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bfmri {

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11). Counter words:
//   x = site (lattice-linear voxel * 4 + slot; slot 0..2 edge +x/+y/+z, 3 the voxel),
//   y = sub (normal pair index / Gamma attempt), z = draw counter, w = tag << 24 | stream.
// ---------------------------------------------------------------------------------------
enum : uint32_t { TAG_W = 1, TAG_A = 2, TAG_LAMBDA = 3, TAG_ALPHA = 4, TAG_BETA = 5, TAG_PROBE = 6 };

__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

struct Rng {
  uint32_t k0, k1, counter, c3;
  __device__ __forceinline__ uint4 call(uint32_t site, uint32_t sub) const {
    return philox(make_uint4(site, sub, counter, c3), k0, k1);
  }
};

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return (double)(a >> 5) * 67108864.0 + (double)(b >> 6);
}

// Box-Muller (1958): u1 in (0, 1] from words 0-1, u2 in [0, 1) from words 2-3.
__device__ __forceinline__ void normal_pair(uint4 w, double& z0, double& z1) {
  const double u1 = (u53(w.x, w.y) + 1.0) * 0x1.0p-53;
  const double u2 = u53(w.z, w.w) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// D normals of one site: lane k from call sub = k / 2, Box-Muller output k % 2.
template <int D>
__device__ __forceinline__ void site_normals(const Rng& g, uint32_t site, double* z) {
#pragma unroll
  for (int j = 0; j < (D + 1) / 2; ++j) {
    double a, b;
    normal_pair(g.call(site, (uint32_t)j), a, b);
    z[2 * j] = a;
    if (2 * j + 1 < D) z[2 * j + 1] = b;
  }
}

// Rademacher sign of lane k: top bit of word k % 4 of call sub = k / 4 (set -> -1).
template <int D>
__device__ __forceinline__ void site_rademacher(const Rng& g, uint32_t site, double* z) {
#pragma unroll
  for (int j = 0; j < (D + 3) / 4; ++j) {
    const uint4 w = g.call(site, (uint32_t)j);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (4 * j + i < D) z[4 * j + i] = (ws[i] >> 31) ? -1.0 : 1.0;
  }
}

// Gamma(shape, scale) by Marsaglia & Tsang (2000) with the exact log test, 8 attempts
// (attempt a: normal from sub 2a, uniform from sub 2a+1), boost u^(1/c) for shape < 1
// (uniform from sub 16). Returns the draw; *exhausted = 1 if no attempt was accepted.
__device__ __forceinline__ double gamma_draw(const Rng& g, uint32_t site, double shape,
                                             double scale, int* exhausted) {
  const bool boost = shape < 1.0;
  const double cp = boost ? shape + 1.0 : shape;
  const double d = cp - 1.0 / 3.0;
  const double cc = 1.0 / sqrt(9.0 * d);
  double res = d;
  bool done = false;
  for (int a = 0; a < 8 && !done; ++a) {
    double x, unused;
    normal_pair(g.call(site, 2u * a), x, unused);
    const uint4 w = g.call(site, 2u * a + 1u);
    const double u = (u53(w.x, w.y) + 1.0) * 0x1.0p-53;
    const double v = 1.0 + cc * x;
    if (v > 0.0) {
      const double v3 = v * v * v;
      if (log(u) < 0.5 * x * x + d - d * v3 + d * log(v3)) {
        res = d * v3;
        done = true;
      }
    }
  }
  *exhausted = done ? 0 : 1;
  if (boost) {
    const uint4 w = g.call(site, 16u);
    const double u = (u53(w.x, w.y) + 1.0) * 0x1.0p-53;
    res *= pow(u, 1.0 / shape);
  }
  return res * scale;
}

// ---------------------------------------------------------------------------------------
// Packed symmetric / lower-triangular D x D blocks, stored as D(D+1)/2 planes of length
// ld (structure of arrays): entry (i, j), i >= j, is plane i(i+1)/2 + j.
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }
__host__ __device__ constexpr int ntri(int d) { return d * (d + 1) / 2; }

template <int D, typename T>
__device__ __forceinline__ void load_packed(const T* __restrict__ base, size_t ld, int n, T* m) {
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) m[e] = base[(size_t)e * ld + n];
}

template <int D, typename T>
__device__ __forceinline__ void store_packed(T* __restrict__ base, size_t ld, int n, const T* m) {
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) base[(size_t)e * ld + n] = m[e];
}

// In-place Cholesky of a packed symmetric matrix; the diagonal is replaced by its inverse.
// Returns false if a pivot is not positive and finite.
template <int D, typename T>
__device__ __forceinline__ bool chol_packed_invdiag(T* m) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T s = m[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= m[tri(j, k)] * m[tri(j, k)];
    ok = ok && (s > T(0)) && (s < T(1e300));
    const T ljj = sqrt(s > T(0) ? s : T(1));
    const T inv = T(1) / ljj;
    m[tri(j, j)] = inv;
#pragma unroll
    for (int i = j + 1; i < D; ++i) {
      T t = m[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= m[tri(i, k)] * m[tri(j, k)];
      m[tri(i, j)] = t * inv;
    }
  }
  return ok;
}

// y = L z with L packed lower, inverted diagonal.
template <int D, typename T>
__device__ __forceinline__ void lower_mul_invdiag(const T* L, const T* z, T* y) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T s = z[i] / L[tri(i, i)];
#pragma unroll
    for (int j = 0; j < i; ++j) s += L[tri(i, j)] * z[j];
    y[i] = s;
  }
}

// z = (L L')^-1 r with L packed lower, inverted diagonal.
template <int D, typename T>
__device__ __forceinline__ void chol_solve_invdiag(const T* L, const T* r, T* z) {
  T y[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T s = r[i];
#pragma unroll
    for (int j = 0; j < i; ++j) s -= L[tri(i, j)] * y[j];
    y[i] = s * L[tri(i, i)];
  }
#pragma unroll
  for (int i = D - 1; i >= 0; --i) {
    T s = y[i];
#pragma unroll
    for (int j = i + 1; j < D; ++j) s -= L[tri(j, i)] * z[j];
    z[i] = s * L[tri(i, i)];
  }
}

// q = B p with B packed symmetric.
template <int D, typename T, typename U>
__device__ __forceinline__ void sym_mul(const T* B, const U* p, U* q) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    U s = U(0);
#pragma unroll
    for (int j = 0; j < D; ++j) s += (U)B[i >= j ? tri(i, j) : tri(j, i)] * p[j];
    q[i] = s;
  }
}

// ---------------------------------------------------------------------------------------
// Bounded grid barrier for cooperative (co-resident) launches. Every wait has a time limit
// read from %globaltimer; on expiry the waiting CTA records BFMRI timeout in *err and
// returns false, and every CTA leaves at its next barrier. The barrier never traps.
// ---------------------------------------------------------------------------------------
struct GridBarrier {
  unsigned int* count;
  unsigned int* gen;
  int* err;                  // 0 = fine; nonzero = error code (sticky)
  unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_acquire_int(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr int ERR_TIMEOUT_CODE = 5;
constexpr int ERR_NOT_SPD_CODE = 3;

__device__ __forceinline__ bool grid_sync(const GridBarrier& b, int* sh_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int g0 = ld_acquire(b.gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(b.count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(b.count, 0u);
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      unsigned int spins = 0;
      while (ld_acquire(b.gen) == g0) {
        if ((++spins & 63u) == 0u) {
          if (ld_acquire_int(b.err) != 0) break;
          if (globaltimer_ns() - t0 > b.timeout_ns) {
            atomicCAS(b.err, 0, ERR_TIMEOUT_CODE);
            break;
          }
        }
      }
    }
    __threadfence();
    *sh_flag = ld_acquire_int(b.err);
  }
  __syncthreads();
  return *sh_flag == 0;
}

// ---------------------------------------------------------------------------------------
// Reducing grid barrier. Every CTA reduces its threads' NV values in a fixed tree and writes
// one row of `part`; the CTA that arrives last sums all rows in a fixed order (independent of
// which CTA it is), publishes the totals in tot[NV] and releases the others, which read them.
// All CTAs therefore obtain bit-identical totals, run after run. Waits are bounded as in
// grid_sync. `sh` needs 32 * NV + NV + 2 doubles of shared memory.
// ---------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ bool grid_allreduce(const GridBarrier& b, double* part, double* tot,
                                               double* v, double* sh, int* sh_int, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* sh_w = sh;                 // [32][NV]
  double* sh_out = sh + 32 * NV;     // [NV]
#pragma unroll
  for (int i = 0; i < NV; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sh_w[warp * NV + i] = v[i];
  }
  __syncthreads();
  const unsigned int nblocks = gridDim.x;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh_w[w * NV + i];
      part[(size_t)blockIdx.x * NV + i] = s;
    }
    const unsigned int g0 = ld_acquire(b.gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(b.count, 1u);
    sh_int[0] = (arrived == nblocks - 1) ? 1 : 0;
    sh_int[1] = (int)g0;
  }
  __syncthreads();
  if (sh_int[0]) {
    // last CTA: fixed-order total of all rows
    if (warp == 0) {
      __threadfence();
      double acc[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = 0.0;
      for (unsigned int r = lane; r < nblocks; r += 32) {
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += __ldcg(part + (size_t)r * NV + i);
      }
#pragma unroll
      for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          sh_out[i] = acc[i];
          tot[i] = acc[i];
        }
        __threadfence();
        atomicExch(b.count, 0u);
        __threadfence();
        atomicAdd(b.gen, 1u);
        sh_int[1] = ld_acquire_int(b.err);
      }
    }
  } else if (threadIdx.x == 0) {
    const unsigned int g0 = (unsigned int)sh_int[1];
    const unsigned long long t0 = globaltimer_ns();
    unsigned int spins = 0;
    bool ok = true;
    while (ld_acquire(b.gen) == g0) {
      if ((++spins & 63u) == 0u) {
        if (ld_acquire_int(b.err) != 0) { ok = false; break; }
        if (globaltimer_ns() - t0 > b.timeout_ns) {
          atomicCAS(b.err, 0, ERR_TIMEOUT_CODE);
          ok = false;
          break;
        }
      }
    }
    __threadfence();
#pragma unroll
    for (int i = 0; i < NV; ++i) sh_out[i] = ok ? __ldcg(tot + i) : 0.0;
    sh_int[1] = ok ? ld_acquire_int(b.err) : 1;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = sh_out[i];
  const bool good = sh_int[1] == 0;
  __syncthreads();
  return good;
}

// ---------------------------------------------------------------------------------------
// Deterministic grid reductions of NV doubles: each CTA reduces its threads' values in a
// fixed tree and writes one row of `part`; after the barrier every CTA re-reduces all rows in
// the same fixed order, so every CTA (and every run) obtains bit-identical sums.
// ---------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_partial(double* v, double* sh /* [32][NV] */, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[warp * NV + i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[w * NV + i];
      part[(size_t)blockIdx.x * NV + i] = s;
    }
  }
  __syncthreads();
}

// After the barrier: all threads get the grid totals.
template <int NV>
__device__ __forceinline__ void grid_total(const double* part, double* sh /* [NV] */, double* out) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] += __ldcg(part + (size_t)b * NV + i);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) sh[i] = acc[i];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = sh[i];
  __syncthreads();
}

}  // namespace bfmri
