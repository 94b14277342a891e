// Sufficient statistics on the tensor cores (tcgen05) for single-precision time series.
//
// The lagged cross-products of Appendix A are, over the common window s = P..T-1-P of the
// lag-difference form, a dense product
//     C[n][(d, k)] = sum_s y_s[n] x_{s+d, k},      d = -P..P,
// of the N x T series with the T x K(2P+1) shifted design. The method needs it to FP64
// accuracy (the A system and RSS cancel lagged sums of size T * 100^2), so the product is
// taken exactly on BF16 tensor cores by splitting both operands into integer digits
// (Ozaki et al., "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012):
//   x_{t,k} = 2^{E_k} sum_i a_i(t, k) 64^{-(i+1)},  y_s[n] = 2^{F_n} sum_j b_j(s, n) 64^{-(j+1)},
// with integer digits |a_i|, |b_j| <= 63 (exact in BF16), E_k a column exponent of X and F_n a
// voxel exponent of Y. Every digit product is an integer below 2^12, and the products of one
// level l = i + j (at most eight digit pairs) summed over at most 512 time steps stay below
// 2^24, so an FP32 accumulator holds each level's sum exactly. Levels 0..7 are kept (the
// next level is below 2^-48 of the leading term), each in its own TMEM accumulator, and are
// combined in FP64 after every window of 512 time steps. Eight digits of Y represent an FP32
// value exactly unless it is below 2^-24 of its voxel's largest value.
//
// Operands: the tile's 128 voxels are the MMA's M rows (A: Y digits, K-major, written by the
// converter warps into shared memory); the columns are (d, k) pairs (B: X digits). All 2P+1
// shifts of X come from one time-major buffer: column group g = d + P of the B operand starts
// g rows further, so the MN-major descriptor's column-group stride is one 16-byte row.
// The X digits are loaded once per CTA by bulk (TMA engine) copies. The terms outside the
// common window (at most P per lag pair and side) and the y'y products stay in FP64 on the
// CUDA cores, computed from the same registers.
#include <climits>
#include <cstring>
#include <vector>

#include "model.cuh"
#include "tc.cuh"

namespace bfmri {

namespace {

constexpr int TC_TILE = 128;       // voxels per tile (MMA M)
constexpr int TC_KS = 16;          // time steps per MMA (K of kind::f16)
constexpr int TC_J = 8;            // digits of Y
constexpr int TC_LEVELS = 8;       // digit levels kept
constexpr int TC_WIN = 512;        // time steps per exact FP32 accumulation window
constexpr int TC_THREADS = 288;    // 8 converter warps + 1 MMA warp
constexpr int YSLICE = TC_TILE * TC_KS * 2;   // bytes of one digit slice of a 16-step chunk
constexpr int YSTAGE = TC_J * YSLICE;         // one pipeline stage

struct TcCtl {
  uint64_t full[2], empty[2], accf, acce, xload;
  uint32_t tmem;
  int err;
  float ymax[2][TC_TILE];
  double syy[TC_TILE][PMAX + 1];
  double xbl[2 * PMAX][16];   // X rows 0 .. 2P-1 (terms before the common window)
  double xbr[2 * PMAX][16];   // X rows T-2P .. T-1 (terms after it)
};

__device__ __forceinline__ void named_sync_converters() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ uint32_t bf16_of_int(float d) { return __float_as_uint(d) >> 16; }

// Knuth's TwoSum: a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// (s, c) += a * b with the product split exactly (p + pe, by a fused multiply-add) and the
// pair renormalised after every term: s + c carries the sum to about 2^-48 of its size.
__device__ __forceinline__ void ff_add_prod(float a, float b, float& s, float& c) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  float t, e;
  two_sum(s, p, t, e);
  two_sum(t, c + (e + pe), s, c);
}

__host__ __device__ inline size_t align1024(size_t b) { return (b + 1023) & ~size_t(1023); }

}  // namespace

size_t stats_tc_smem_bytes(int T, int K, int P, int I) {
  const int Tw = T - 2 * P;
  const int nk = (Tw + TC_KS - 1) / TC_KS;
  const int Tpad = TC_KS * nk + 8;
  const int groups = (K + 7) / 8;
  return align1024((size_t)groups * I * Tpad * 16) + 2 * (size_t)YSTAGE + sizeof(TcCtl);
}

// Digits of X for the tensor-core statistics: dig[((g I + i) Tpad + u) 8 + kk] holds digit i
// of x_{u, 8g + kk} (BF16 bits; zero outside 0 <= u < T, k < K), exps[k] = E_k with
// |x_{u,k}| < 2^{E_k}.
void stats_tc_digits(const double* X, int T, int K, int P, int I, std::vector<uint16_t>& dig,
                     std::vector<int>& exps, int& Tpad) {
  const int Tw = T - 2 * P;
  Tpad = TC_KS * ((Tw + TC_KS - 1) / TC_KS) + 8;
  const int groups = (K + 7) / 8;
  dig.assign((size_t)groups * I * Tpad * 8, 0);
  exps.assign(K, 0);
  for (int k = 0; k < K; ++k) {
    double m = 0.0;
    for (int u = 0; u < T; ++u) m = std::max(m, std::fabs(X[u + (size_t)T * k]));
    exps[k] = m > 0.0 ? std::ilogb(m) + 1 : 0;
    const int g = k / 8, kk = k % 8;
    for (int u = 0; u < T; ++u) {
      double v = std::ldexp(X[u + (size_t)T * k], -exps[k]);
      for (int i = 0; i < I; ++i) {
        v *= 64.0;
        const double d = std::trunc(v);
        v -= d;
        const float df = (float)d;
        uint32_t bits;
        std::memcpy(&bits, &df, 4);
        dig[(((size_t)g * I + i) * Tpad + u) * 8 + kk] = (uint16_t)(bits >> 16);
      }
    }
  }
}

template <int NMMA>
__global__ void __launch_bounds__(TC_THREADS, 1) k_stats_tc(StatsTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int T = a.T, P = a.P, K = a.K, N = a.N, I = a.I, Tpad = a.Tpad, NG = a.groups;
  const int Tw = T - 2 * P;
  const size_t xs_bytes = (size_t)NG * I * Tpad * 16;
  unsigned char* xs = smem;
  unsigned char* yb = smem + align1024(xs_bytes);
  TcCtl* c = reinterpret_cast<TcCtl*>(yb + 2 * YSTAGE);
  constexpr uint32_t TCOLS = NMMA * TC_LEVELS <= 128 ? 128u : (NMMA * TC_LEVELS <= 256 ? 256u : 512u);
  constexpr uint32_t IDESC = tc::idesc_bf16_f32(TC_TILE, NMMA, false, true);
  constexpr int HALF = NMMA / 2;          // accumulator columns per converter group
  constexpr int PC = NMMA / 16 - 1;       // the AR order this instance serves (a.P == PC)
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&c->full[b], 128);
      tc::mbar_init(&c->empty[b], 1);
    }
    tc::mbar_init(&c->accf, 1);
    tc::mbar_init(&c->acce, 256);
    tc::mbar_init(&c->xload, 1);
    c->err = 0;
    tc::mbar_init_fence();
  }
  if (warp == 8) tc::tmem_alloc(&c->tmem, TCOLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = c->tmem;
  // the X digits, once per CTA, by bulk copies
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&c->xload, (uint32_t)xs_bytes);
    for (size_t off = 0; off < xs_bytes; off += 32768) {
      const uint32_t nb = (uint32_t)(xs_bytes - off < 32768 ? xs_bytes - off : 32768);
      tc::bulk_g2s(xs + off, reinterpret_cast<const unsigned char*>(a.xdig) + off, nb, &c->xload);
    }
  }
  if (!tc::mbar_wait(&c->xload, 0)) atomicExch(&c->err, 1);
  for (int i = tid; i < 2 * P * K; i += blockDim.x) {
    const int t = i / K, k = i % K;
    c->xbl[t][k] = __ldg(a.X + t + (size_t)T * k);
    c->xbr[t][k] = __ldg(a.X + (T - 2 * P + t) + (size_t)T * k);
  }
  __syncthreads();

  const bool conv = warp < 8;
  const int h = warp >> 2;                  // converter group: 0 or 1
  const int row = 32 * (warp & 3) + lane;   // voxel row of the tile = TMEM lane
  const int ntiles = (N + TC_TILE - 1) / TC_TILE;
  uint32_t gstep = 0;                       // 16-step chunks issued so far (same on all threads)
  uint32_t wins = 0;                        // accumulator windows completed
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = tile * TC_TILE + row;
    const bool valid = conv && n < N;
    int Fv = 0;   // voxel exponent: |y_s| < 2^Fv over the window
    if (conv) {
      float m = 0.f;
      const int mid = P + Tw / 2;
      const int s_lo = h == 0 ? P : mid, s_hi = h == 0 ? mid : T - P;
      if (valid) {
        int s = s_lo;
        for (; s + 8 <= s_hi; s += 8) {
          float v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = __ldg(a.Y + (size_t)(s + i) * N + n);
#pragma unroll
          for (int i = 0; i < 8; ++i) m = fmaxf(m, fabsf(v[i]));
        }
        for (; s < s_hi; ++s) m = fmaxf(m, fabsf(__ldg(a.Y + (size_t)s * N + n)));
      }
      c->ymax[h][row] = m;
      named_sync_converters();
      const float mm = fmaxf(c->ymax[0][row], c->ymax[1][row]);
      Fv = mm > 0.f ? ilogbf(mm) + 1 : 0;
    }
    // the series values the terms outside the common window use: y_0 .. y_{2P-1} and
    // y_{T-P} .. y_{T-1}
    float ybl[2 * PMAX], ybr[PMAX];
#pragma unroll
    for (int t = 0; t < 2 * PMAX; ++t) ybl[t] = (valid && t < 2 * PC) ? __ldg(a.Y + (size_t)t * N + n) : 0.f;
#pragma unroll
    for (int i = 0; i < PMAX; ++i) ybr[i] = (valid && i < PC) ? __ldg(a.Y + (size_t)(T - PC + i) * N + n) : 0.f;
    // y * 2^-Fv by one multiplication while 2^-Fv is a normal number, else by ldexpf
    const bool plain_scale = Fv >= -125 && Fv <= 125;
    const float scale = plain_scale ? __int_as_float((127 - Fv) << 23) : 1.f;
    double syy[PMAX + 1];
#pragma unroll
    for (int e = 0; e <= PMAX; ++e) syy[e] = 0.0;
    for (int kg = 0; kg < NG; ++kg) {
      for (int w0 = 0; w0 < Tw; w0 += TC_WIN) {
        const int span = Tw - w0 < TC_WIN ? Tw - w0 : TC_WIN;
        const int nsteps = (span + TC_KS - 1) / TC_KS;
        if (warp == 8) {
          if (lane == 0) {
            if (wins > 0 && !tc::mbar_wait(&c->acce, (wins - 1) & 1)) atomicExch(&c->err, 2);
            tc::fence_after_sync();
            for (int q = 0; q < nsteps; ++q) {
              const uint32_t g = gstep + q, b = g & 1, u = g >> 1;
              if (!tc::mbar_wait(&c->full[b], u & 1)) atomicExch(&c->err, 3);
              tc::fence_after_sync();
              const int s0 = P + w0 + TC_KS * q;
              uint64_t ad[TC_J];
#pragma unroll
              for (int j = 0; j < TC_J; ++j)
                ad[j] = tc::smem_desc(tc::smem_u32(yb + b * YSTAGE + j * YSLICE), 128, 256);
              for (int l = 0; l < TC_LEVELS; ++l) {
                const int imax = l < I - 1 ? l : I - 1;
                for (int i = 0; i <= imax; ++i) {
                  const int j = l - i;
                  if (j >= TC_J) continue;
                  const uint64_t bd = tc::smem_desc(
                      tc::smem_u32(xs + (((size_t)kg * I + i) * Tpad + (s0 - P)) * 16), 128, 16);
                  tc::mma_bf16(tbase + (uint32_t)(l * NMMA), ad[j], bd, IDESC, q > 0 || i > 0);
                }
              }
              tc::mma_commit(&c->empty[b]);
            }
            tc::mma_commit(&c->accf);
          }
          __syncwarp();
        } else {
          for (int q = 0; q < nsteps; ++q) {
            const uint32_t g = gstep + q, b = g & 1, u = g >> 1;
            if ((int)b != h) continue;
            if (u >= 1 && !tc::mbar_wait(&c->empty[b], (u - 1) & 1)) atomicExch(&c->err, 4);
            const int s0 = P + w0 + TC_KS * q;
            float y[TC_KS + PMAX];
#pragma unroll
            for (int t = 0; t < TC_KS + PMAX; ++t) {
              const int s = s0 + t;
              y[t] = (valid && s < T) ? __ldg(a.Y + (size_t)s * N + n) : 0.f;
            }
            uint32_t w[TC_J][TC_KS / 2];
#pragma unroll
            for (int t = 0; t < TC_KS; ++t) {
              float v = (s0 + t < T - P) ? (plain_scale ? y[t] * scale : ldexpf(y[t], -Fv)) : 0.f;
#pragma unroll
              for (int j = 0; j < TC_J; ++j) {
                v *= 64.f;
                const float d = truncf(v);
                v -= d;
                const uint32_t bits = bf16_of_int(d);
                if (t & 1) w[j][t >> 1] |= bits << 16;
                else w[j][t >> 1] = bits;
              }
            }
            unsigned char* base = yb + b * YSTAGE + (row >> 3) * 256 + (row & 7) * 16;
#pragma unroll
            for (int j = 0; j < TC_J; ++j) {
              uint4* p0 = reinterpret_cast<uint4*>(base + j * YSLICE);
              uint4* p1 = reinterpret_cast<uint4*>(base + j * YSLICE + 128);
              *p0 = make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
              *p1 = make_uint4(w[j][4], w[j][5], w[j][6], w[j][7]);
            }
            if (kg == 0 && valid) {
              // y'y products of the chunk: exact FP32 product splits summed as float pairs,
              // then one FP64 addition per lag and chunk
#pragma unroll
              for (int e = 0; e <= PMAX; ++e) {
                if (e <= P) {
                  float hi = 0.f, lo = 0.f;
#pragma unroll
                  for (int t = 0; t < TC_KS; ++t)
                    if (s0 + t < T - P) ff_add_prod(y[t], y[t + e], hi, lo);
                  syy[e] += (double)hi + (double)lo;
                }
              }
            }
            tc::fence_async_smem();
            tc::mbar_arrive(&c->full[b]);
          }
          // this window's levels -> FP64 (each level's FP32 sum is an exact integer)
          if (!tc::mbar_wait(&c->accf, wins & 1)) atomicExch(&c->err, 5);
          tc::fence_after_sync();
          const uint32_t lane_base = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
          // Each level's sum is an integer below 2^24; levels 0..3 and 4..7 combine exactly
          // in 64-bit integers (sum_l L_l 64^(3-l) < 2^43), and only the two results are
          // converted: value = 2^-18 hi + 2^-42 lo in units of level 0.
          // Windows before the last keep their partial sums in the output plane of the pair
          // (p0, p0 - d), p0 = max(d, 0), which the last window reads back and overwrites.
          const bool first_win = w0 == 0, last_win = w0 + TC_WIN >= Tw;
          const size_t ld = a.ld;
#pragma unroll
          for (int cc = 0; cc < HALF / 8; ++cc) {
            uint32_t v[TC_LEVELS][8];
#pragma unroll
            for (int l = 0; l < TC_LEVELS; ++l)
              tc::tmem_ld8(lane_base + (uint32_t)(l * NMMA + h * HALF + cc * 8), v[l]);
            tc::tmem_wait_ld();
            const int gsh = (h * HALF + cc * 8) >> 3, d = gsh - PC;
            if (!valid || gsh > 2 * PC) continue;
            const int p0 = d > 0 ? d : 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int k = 8 * kg + e;
              if (k >= K) continue;
              long long hi = 0, lo = 0;
#pragma unroll
              for (int l = 0; l < 4; ++l) {
                hi = hi * 64 + (long long)__float2int_rz(__uint_as_float(v[l][e]));
                lo = lo * 64 + (long long)__float2int_rz(__uint_as_float(v[l + 4][e]));
              }
              double acc = __ll2double_rn(hi) * 0x1p-18 + __ll2double_rn(lo) * 0x1p-42;
              double* tmp = a.stats + sxy_plane(p0, p0 - d, k, K, PC) * ld + n;
              if (!first_win) acc += *tmp;
              if (!last_win) {
                *tmp = acc;
                continue;
              }
              // Sxy of the pairs (p, q = p - d): the window sum scaled back, plus the terms
              // t = P-p .. P-1 before the window (added as p grows) and t = T-P .. T-1-p after it
              const double C = ldexp(acc, a.xexp[k] + Fv - 12);
              double after[PC + 1];
#pragma unroll
              for (int pp = 0; pp <= PC; ++pp) {
                double w = 0.0;
#pragma unroll
                for (int i = 0; i <= PC - 1 - pp; ++i) w += (double)ybr[i] * c->xbr[PC + i + d][k];
                after[pp] = w;
              }
              double before = 0.0;
#pragma unroll
              for (int pp = 0; pp <= PC; ++pp) {
                if (pp >= 1) before += (double)ybl[PC - pp] * c->xbl[PC - pp + d][k];
                if (pp >= d && pp - d <= PC)
                  a.stats[sxy_plane(pp, pp - d, k, K, PC) * ld + n] = C + before + after[pp];
              }
            }
          }
          tc::fence_before_sync();
          tc::mbar_arrive(&c->acce);
        }
        gstep += nsteps;
        wins += 1;
      }
    }
    // Syy: the two groups' window sums, plus the boundary terms
    if (conv) {
      if (h == 1) {
#pragma unroll
        for (int e = 0; e <= PMAX; ++e) c->syy[row][e] = syy[e];
      }
      named_sync_converters();
      if (h == 0 && valid) {
        const size_t ld = a.ld;
#pragma unroll
        for (int e = 0; e <= PC; ++e) {
          const double cyy = syy[e] + c->syy[row][e];
#pragma unroll
          for (int q = e; q <= PC; ++q) {
            double v = cyy;
#pragma unroll
            for (int j = 1; j <= q; ++j) v += (double)ybl[PC - j] * (double)ybl[PC - j + e];   // t = P - j
#pragma unroll
            for (int i = 0; i <= PC - 1 - q; ++i) v += (double)ybr[i] * (double)ybr[i + e];    // t = T - P + i
            a.stats[(size_t)syy_index(q - e, q, PC) * ld + n] = v;
          }
        }
      }
      named_sync_converters();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 8) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, TCOLS);
  }
  if (tid == 0 && c->err != 0) atomicExch(a.err, c->err);
}

namespace {

template <int NMMA>
cudaError_t stats_tc_n(const StatsTcArgs& a, size_t smem, cudaStream_t s) {
  const void* kern = (const void*)k_stats_tc<NMMA>;
  cudaError_t e = raise_smem_limit(kern, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (a.sm_cap > 0 && a.sm_cap < nsm) nsm = a.sm_cap;
  const int ntiles = (a.N + TC_TILE - 1) / TC_TILE;
  const int grid = ntiles < nsm ? ntiles : nsm;
  k_stats_tc<NMMA><<<grid, TC_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool stats_tc_supported(int T, int K, int P, int* I_out) {
  if (P > 3 || K < 1 || K > 16 || T - 2 * P < 1) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  for (int I = 8; I >= 7; --I) {
    if (stats_tc_smem_bytes(T, K, P, I) <= (size_t)optin) {
      if (I_out) *I_out = I;
      return true;
    }
  }
  return false;
}

cudaError_t launch_stats_tc(const StatsTcArgs& a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  // at least 120 KB of shared memory: one CTA per SM, so no two CTAs contend for TMEM
  size_t smem = stats_tc_smem_bytes(a.T, a.K, a.P, a.I);
  if (smem < (size_t)120 * 1024) smem = (size_t)120 * 1024;
  switch (a.P) {
    case 0: return stats_tc_n<16>(a, smem, s);
    case 1: return stats_tc_n<32>(a, smem, s);
    case 2: return stats_tc_n<48>(a, smem, s);
    case 3: return stats_tc_n<64>(a, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfmri
