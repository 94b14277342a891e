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
enum : uint32_t { TAG_W = 1, TAG_A = 2, TAG_LAMBDA = 3, TAG_ALPHA = 4, TAG_BETA = 5, TAG_PROBE = 6,
                  TAG_ALPHA_PROP = 7,   // anisotropic prior: proposal normals, acceptance uniform
                  TAG_ALPHA_AUX = 8 };  // anisotropic prior: the auxiliary draw's edge normals

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

// Philox key (k0, k1) and the counter words: (site, sub, draw counter, c3). The draw counter
// is `counter`, plus the device word *dctr when dctr is set (a captured CUDA graph replays one
// sweep for every draw counter: the graph advances the device word, not a kernel argument).
struct Rng {
  uint32_t k0, k1, counter, c3;
  const uint32_t* dctr;
  __device__ __forceinline__ uint4 call(uint32_t site, uint32_t sub) const {
    const uint32_t c = dctr ? counter + __ldg(dctr) : counter;
    return philox(make_uint4(site, sub, c, c3), k0, k1);
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
// Asynchronous global -> shared copies (cp.async): the copy completes in the background and
// cp.async.wait_group blocks only this thread until its own earlier groups have landed.
// A false predicate copies nothing and fills the destination with zeros.
// ---------------------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  const int src_size = pred ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(s), "l"(gsrc), "n"(BYTES), "r"(src_size)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

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

// 1/sqrt(s) for s > 0 by Newton's iteration for the reciprocal square root,
// y <- y + y (1 - s y^2) / 2, from the hardware's approximate FP64 value: each step squares
// the relative error, and two steps take it to the FP64 rounding level. Far fewer FP64
// instructions than a correctly rounded square root followed by a division, which matters on
// a part whose FP64 issue rate is 2 lanes per clock per SM.
__device__ __forceinline__ double rsqrt_nr(double s) {
  double y;
  asm("rsqrt.approx.f64 %0, %1;" : "=d"(y) : "d"(s));
  double h = fma(-s * y, y, 1.0);
  y = fma(0.5 * y, h, y);
  h = fma(-s * y, y, 1.0);
  return fma(0.5 * y, h, y);
}

// In-place Cholesky of a packed symmetric matrix; the diagonal is replaced by its inverse and,
// if diag is given, the pivots' square roots l_jj are written there. Returns false if a pivot
// is not positive and finite.
template <int D, typename T>
__device__ __forceinline__ bool chol_packed_invdiag(T* m, T* diag = nullptr) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    T s = m[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= m[tri(j, k)] * m[tri(j, k)];
    ok = ok && (s > T(0)) && (s < T(1e300));
    const T sp = s > T(0) ? s : T(1);
    T ljj, inv;
    if constexpr (sizeof(T) == 8) {
      inv = rsqrt_nr(sp);
      ljj = sp * inv;
    } else {
      ljj = sqrt(sp);
      inv = T(1) / ljj;
    }
    if (diag) diag[j] = ljj;
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

// y = L z with L packed lower and its diagonal l_jj given separately (no division).
template <int D, typename T>
__device__ __forceinline__ void lower_mul_diag(const T* L, const T* diag, const T* z, T* y) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T s = z[i] * diag[i];
#pragma unroll
    for (int j = 0; j < i; ++j) s += L[tri(i, j)] * z[j];
    y[i] = s;
  }
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
// Bounded grid barrier for cooperative (co-resident) launches. The host zeroes the arrival
// counter (and the generation word) before every cooperative launch (reset_grid_barrier);
// during the launch the counter only grows. Thread 0 of every CTA arrives with a release
// reduction on it, which needs no round trip, and barrier j of the launch (0-based) is passed
// once the counter reaches (j + 1) x gridDim.x, which thread 0 polls with acquire loads. The
// generation word is released only by the multi-RHS reducing barrier, whose last CTA to
// arrive does scalar work before the others may go on. Every wait has a time limit read
// from %globaltimer: on expiry the CTA records a timeout in *err and returns false, and
// every CTA leaves at its next barrier. The barrier never traps.
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

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void red_add_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr int ERR_TIMEOUT_CODE = 5;
constexpr int ERR_NOT_SPD_CODE = 3;
constexpr int ERR_LAYOUT_CODE = 11;   // a kernel found its launch layout inconsistent with its data

// The number of barriers this CTA has passed in the current launch (thread 0's copy). Every
// kernel that uses the barriers below calls grid_barrier_start first; the counter it pairs
// with was zeroed by the host before the launch.
static __shared__ unsigned int g_bar_gen;

__device__ __forceinline__ void grid_barrier_start(const GridBarrier&) {
  if (threadIdx.x == 0) g_bar_gen = 0u;
}

// Raises the dynamic shared-memory limit of kernel `kern` on the current device to at least
// `bytes` and never lowers it. The limit is a property of the function, shared by every host
// thread that launches it (the server's slots run launchers concurrently); setting it to each
// call's own size could lower it between another thread's set and that thread's launch, which
// then fails. Returns the error of the attribute call, cudaSuccess when no change is needed.
cudaError_t raise_smem_limit(const void* kern, size_t bytes);

// Zeroes the arrival counter and the generation word; the launchers call it on the launch
// stream before every cooperative launch that uses the barrier.
inline cudaError_t reset_grid_barrier(const GridBarrier& b, cudaStream_t stream) {
  if (b.gen == b.count + 1) return cudaMemsetAsync(b.count, 0, 2 * sizeof(unsigned int), stream);
  cudaError_t e = cudaMemsetAsync(b.count, 0, sizeof(unsigned int), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.gen, 0, sizeof(unsigned int), stream);
  return e;
}

// Polls *w until it has reached target (wrap-safe); false on error or time-out.
__device__ __forceinline__ bool wait_reach(const GridBarrier& b, const unsigned int* w,
                                           unsigned int target) {
  const unsigned long long t0 = globaltimer_ns();
  unsigned int spins = 0;
  while ((int)(ld_acquire(w) - target) < 0) {
    if ((++spins & 255u) == 0u) {
      if (ld_acquire_int(b.err) != 0) return false;
      if (globaltimer_ns() - t0 > b.timeout_ns) {
        atomicCAS(b.err, 0, ERR_TIMEOUT_CODE);
        return false;
      }
    }
  }
  return true;
}

// Arrival of this CTA at barrier g0 of the launch and the wait for all others (thread 0).
__device__ __forceinline__ bool arrive_and_wait(const GridBarrier& b, unsigned int g0) {
  red_add_release(b.count, 1u);
  return wait_reach(b, b.count, (g0 + 1u) * gridDim.x);
}

__device__ __forceinline__ bool grid_sync(const GridBarrier& b, int* sh_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g0 = g_bar_gen;
    const bool ok = arrive_and_wait(b, g0);
    g_bar_gen = g0 + 1u;
    *sh_flag = ok ? 0 : 1;
  }
  __syncthreads();
  return *sh_flag == 0;
}

// ---------------------------------------------------------------------------------------
// Warp reduction of 4 doubles with 6 FP64 additions per warp instead of 20 (FP64 issue is
// scarce on this part): the first two exchange levels split the values between lane halves
// and quarters, the last three are a plain butterfly. Afterwards value j is complete in
// lanes [8j, 8j + 8).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_reduce4(const double* v) {
  const int l = threadIdx.x & 31;
  const bool hi16 = (l & 16) != 0;
  const double a_keep = hi16 ? v[2] : v[0], b_keep = hi16 ? v[3] : v[1];
  const double a_send = hi16 ? v[0] : v[2], b_send = hi16 ? v[1] : v[3];
  const double a = a_keep + __shfl_xor_sync(0xffffffffu, a_send, 16);
  const double b = b_keep + __shfl_xor_sync(0xffffffffu, b_send, 16);
  const bool hi8 = (l & 8) != 0;
  double c = (hi8 ? b : a) + __shfl_xor_sync(0xffffffffu, hi8 ? a : b, 8);
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

// Block totals of 4 doubles per thread, fixed order; every thread receives them in out.
// sh needs 4 * 32 + 4 doubles.
__device__ __forceinline__ void block_reduce4(const double* v, double* sh, double* out) {
  const int l = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double c = warp_reduce4(v);
  if ((l & 7) == 0) sh[warp * 4 + (l >> 3)] = c;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    const int j = l & 3;
    double acc = 0.0;
    for (int w = l >> 2; w < nw; w += 8) acc += sh[w * 4 + j];
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (l < 4) sh[128 + l] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = sh[128 + i];
}

// ---------------------------------------------------------------------------------------
// Reducing grid barrier over 4 doubles. Every CTA writes its block totals to one row of a
// partial buffer and arrives at the barrier; once all have arrived, every CTA sums all rows
// itself in the same fixed order, so all obtain bit-identical totals, run after run, with no
// second publication round after the barrier. The two row buffers alternate with the barrier
// generation: back-to-back reductions (generations g and g + 1) write different buffers, and
// two reductions that write the same buffer have at least one barrier between them, which no
// CTA passes before every CTA has read the earlier rows. part0 and part1 hold gridDim.x rows
// of 4 doubles each. sh needs 4 * 32 + 8 doubles, sh_int 2 ints.
// ---------------------------------------------------------------------------------------
// Sums the rows of a partial buffer that every CTA wrote before a barrier this CTA has
// passed, in a fixed order, so every CTA obtains bit-identical totals; every thread receives
// them in out. sh needs 4 * 32 + 8 doubles. With at least 128 threads, warps w0 .. w0 + 3
// (w0 + 4 <= the CTA's warps) do the loads, so a caller may hand them to warps that are idle
// at that point; the summation order, and so the totals, do not depend on w0.
__device__ __forceinline__ void allreduce4_collect(const double* part, double* sh, double* out,
                                                   int w0 = 0) {
  const int l = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int nblocks = gridDim.x;
  double* sh_out = sh + 132;
  if (blockDim.x >= 128) {
    // warp w0 + j sums value j: lane l over rows l + 32 i (5 rows per lane and round, as a
    // fixed pairwise tree), then a butterfly; the four warps run on different SM sub-partitions
    const int j = warp - w0;
    if (j >= 0 && j < 4) {
      constexpr int RU = 5;
      double acc = 0.0;
      for (unsigned int r0 = (unsigned int)l; r0 < nblocks; r0 += 32u * RU) {
        double buf[RU];
#pragma unroll
        for (int i = 0; i < RU; ++i) {
          const unsigned int r = r0 + 32u * i;
          buf[i] = r < nblocks ? __ldcg(part + (size_t)r * 4 + j) : 0.0;
        }
        acc += ((buf[0] + buf[1]) + (buf[2] + buf[3])) + buf[4];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (l == 0) sh_out[j] = acc;
    }
  } else if (warp == 0) {
    // lane l sums value (l & 3) over rows (l >> 2) + 8 i (20 rows per lane and round)
    const int j = l & 3;
    constexpr int RU = 20;
    double acc = 0.0;
    for (unsigned int r0 = (unsigned int)(l >> 2); r0 < nblocks; r0 += 8u * RU) {
      double buf[RU];
#pragma unroll
      for (int i = 0; i < RU; ++i) {
        const unsigned int r = r0 + 8u * i;
        buf[i] = r < nblocks ? __ldcg(part + (size_t)r * 4 + j) : 0.0;
      }
#pragma unroll
      for (int w = 1; w < RU; w *= 2)
#pragma unroll
        for (int i = 0; i + w < RU; i += 2 * w) buf[i] += buf[i + w];
      acc += buf[0];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (l < 4) sh_out[l] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = sh_out[i];
  __syncthreads();
}

__device__ __forceinline__ bool grid_allreduce4(const GridBarrier& b, double* part0, double* part1,
                                                const double* v, double* sh, int* sh_int, double* out) {
  double bt[4];
  block_reduce4(v, sh, bt);
  if (threadIdx.x == 0) {
    const unsigned int g0 = g_bar_gen;
    double* part = (g0 & 1u) ? part1 : part0;
#pragma unroll
    for (int i = 0; i < 4; ++i) part[(size_t)blockIdx.x * 4 + i] = bt[i];
    const bool ok = arrive_and_wait(b, g0);
    g_bar_gen = g0 + 1u;
    sh_int[0] = ok ? 0 : 1;
    sh_int[1] = (int)(g0 & 1u);
  }
  __syncthreads();
  const bool good = sh_int[0] == 0;
  if (!good) return false;
  allreduce4_collect(sh_int[1] ? part1 : part0, sh, out);
  return true;
}

// Split form: the CTA's block totals of v go to the row buffer of the current barrier
// generation before a plain grid barrier (grid_sync); after that barrier, allreduce4_collect
// on the returned buffer gives the totals. The collection must finish before the CTA arrives
// at the following barrier (the buffers alternate with the generation).
__device__ __forceinline__ const double* allreduce4_post(double* part0, double* part1,
                                                         const double* v, double* sh) {
  double bt[4];
  block_reduce4(v, sh, bt);   // ends with __syncthreads: every thread sees g_bar_gen
  double* part = (g_bar_gen & 1u) ? part1 : part0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) part[(size_t)blockIdx.x * 4 + i] = bt[i];
  }
  return part;
}

// ---------------------------------------------------------------------------------------
// Float-float (double-single) sums for the FP32 inner solves: a value is hi + lo with
// |lo| <= ulp(hi) / 2, about 48 significant bits. Addition is Knuth's TwoSum of the leading
// parts plus the trailing parts, renormalised by Dekker's FastTwoSum. Every step runs on
// the FP32 pipe, whose dependent latency is a small fraction of an FP64 operation's on this
// part, so reduction trees of these pairs finish far sooner than FP64 trees.
// ---------------------------------------------------------------------------------------
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_of(float x) { return FF{x, 0.f}; }

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bv = s - a.hi;
  const float e = (a.hi - (s - bv)) + (b.hi - bv);
  const float t = (a.lo + b.lo) + e;
  const float hi = s + t;
  return FF{hi, t - (hi - s)};
}

__device__ __forceinline__ FF ff_shfl_xor(FF a, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// Reducing grid barrier over 4 float-float values: the same protocol as grid_allreduce4
// (rows alternating with the barrier generation, every CTA summing all rows in a fixed
// order), with the block and cross-CTA sums done in float-float; totals are returned as
// doubles. A row holds 4 (hi, lo) pairs, the size of a grid_allreduce4 row.
// Block totals of 4 float-float values (every warp, then warp 0 over the warps); lane 0 of
// warp 0 holds them in c4 on return. shw needs 4 * 2 floats per warp.
__device__ __forceinline__ void block_reduce4_ff(const FF* v, float* shw, FF* c4) {
  const int l = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwc = (blockDim.x + 31) >> 5;
  FF w4[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    w4[i] = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w4[i] = ff_add(w4[i], ff_shfl_xor(w4[i], o));
  }
  if (l == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      shw[(warp * 4 + i) * 2 + 0] = w4[i].hi;
      shw[(warp * 4 + i) * 2 + 1] = w4[i].lo;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c4[i] = l < nwc ? FF{shw[(l * 4 + i) * 2 + 0], shw[(l * 4 + i) * 2 + 1]} : FF{0.f, 0.f};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c4[i] = ff_add(c4[i], ff_shfl_xor(c4[i], o));
    }
  }
}

// Sums the float-float rows (8 floats each) that every CTA wrote before a barrier this CTA
// has passed, in a fixed order; every thread receives the FP64 totals in out.
// With four warps or more, warps w0 .. w0 + 3 (w0 + 4 <= the CTA's warps) do the loads; the
// summation order, and so the totals, do not depend on w0.
__device__ __forceinline__ void allreduce4_ff_collect(const float* part, double* sh, double* out,
                                                      int w0 = 0) {
  const int l = threadIdx.x & 31;
  const int nwc = (blockDim.x + 31) >> 5;
  const unsigned int nblocks = gridDim.x;
  double* sh_out = sh + 132;
  // warp w0 + j sums value j (warp 0 all four when the CTA has fewer warps) over the rows
  const int nsum = nwc >= 4 ? 4 : 1;
  const int warp = nwc >= 4 ? (int)(threadIdx.x >> 5) - w0 : (int)(threadIdx.x >> 5);
  if (warp >= 0 && warp < nsum) {
    for (int j = warp; j < 4; j += nsum) {
      FF acc{0.f, 0.f};
      for (unsigned int r = (unsigned int)l; r < nblocks; r += 32u) {
        const float2 p = __ldcg(reinterpret_cast<const float2*>(part + (size_t)r * 8 + 2 * j));
        acc = ff_add(acc, FF{p.x, p.y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = ff_add(acc, ff_shfl_xor(acc, o));
      if (l == 0) sh_out[j] = ff_to_double(acc);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = sh_out[i];
  __syncthreads();
}

__device__ __forceinline__ bool grid_allreduce4_ff(const GridBarrier& b, double* part0, double* part1,
                                                   const FF* v, double* sh, int* sh_int, double* out) {
  float* shw = reinterpret_cast<float*>(sh);   // [warp][4][2] floats: 96 floats = 48 doubles
  FF c4[4];
  block_reduce4_ff(v, shw, c4);
  if (threadIdx.x == 0) {
    const unsigned int g0 = g_bar_gen;
    float* row = reinterpret_cast<float*>((g0 & 1u) ? part1 : part0) + (size_t)blockIdx.x * 8;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      row[2 * i + 0] = c4[i].hi;
      row[2 * i + 1] = c4[i].lo;
    }
    const bool ok = arrive_and_wait(b, g0);
    g_bar_gen = g0 + 1u;
    sh_int[0] = ok ? 0 : 1;
    sh_int[1] = (int)(g0 & 1u);
  }
  __syncthreads();
  if (sh_int[0] != 0) return false;
  allreduce4_ff_collect(reinterpret_cast<const float*>(sh_int[1] ? part1 : part0), sh, out);
  return true;
}

// Split form (see allreduce4_post): the CTA's float-float totals go to the row buffer of the
// current barrier generation before a plain grid barrier; collect after it.
__device__ __forceinline__ const float* allreduce4_ff_post(double* part0, double* part1, const FF* v,
                                                           double* sh) {
  float* shw = reinterpret_cast<float*>(sh);
  FF c4[4];
  block_reduce4_ff(v, shw, c4);
  __syncthreads();   // every thread sees g_bar_gen; shw free again
  float* row = reinterpret_cast<float*>((g_bar_gen & 1u) ? part1 : part0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      row[(size_t)blockIdx.x * 8 + 2 * i + 0] = c4[i].hi;
      row[(size_t)blockIdx.x * 8 + 2 * i + 1] = c4[i].lo;
    }
  }
  return row;
}

}  // namespace bfmri
