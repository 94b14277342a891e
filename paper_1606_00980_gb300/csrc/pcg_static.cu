// bfmri_pcg_solve_static: the FP64 PCG solve of bfmri_sample_W for caller-owned device data,
// with all of its scratch memory (preconditioner factor, work vectors, reduction and barrier
// words) in one fixed file-scope device array, so that the call allocates nothing.
//
// Host code must not hand the array's name to a kernel: on the host it is only a stand-in
// symbol. Its device address is looked up once per device with cudaGetSymbolAddress (with
// that device current, on the first call made on it) and cached.
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/bfmri.h"
#include "pcg.cuh"

namespace bfmri {
void set_global_error(const std::string& msg);  // bfmri_api.cu
}

using namespace bfmri;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Block-Jacobi factor chol(B_n + diag(s) deg_n) (inverted diagonal) into the scratch area.
template <int D>
__global__ void k_static_precond(int N, size_t ld, int ndir, const int* nbr, const double* blocks,
                                 const double* scale, size_t lds, double* mfac, int* bad) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double M[ntri(D)];
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) M[e] = blocks[(size_t)e * ld + n];
  int deg = 0;
  for (int d = 0; d < ndir; ++d) deg += nbr[(size_t)d * ld + n] >= 0 ? 1 : 0;
#pragma unroll
  for (int k = 0; k < D; ++k) M[tri(k, k)] += scale[k] * (double)deg;
  if (!chol_packed_invdiag<D>(M)) atomicMin(bad, n);
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) mfac[(size_t)e * lds + n] = M[e];
}

template <int D>
cudaError_t launch_static_precond(int N, size_t ld, int ndir, const int* nbr, const double* blocks,
                                  const double* scale, size_t lds, double* mfac, int* bad,
                                  cudaStream_t s) {
  k_static_precond<D><<<(N + 127) / 128, 128, 0, s>>>(N, ld, ndir, nbr, blocks, scale, lds, mfac, bad);
  return cudaGetLastError();
}

cudaError_t static_precond(int D, int N, size_t ld, int ndir, const int* nbr, const double* blocks,
                           const double* scale, size_t lds, double* mfac, int* bad, cudaStream_t s) {
  switch (D) {
#define CASE(d) case d: return launch_static_precond<d>(N, ld, ndir, nbr, blocks, scale, lds, mfac, bad, s);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

bfmri_status err(bfmri_status code, const std::string& msg) {
  set_global_error("bfmri_pcg_solve_static: " + msg);
  return code;
}

// Device address of the scratch array on the current device (looked up on first use).
bfmri_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(BFMRI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return err(BFMRI_ERR_INTERNAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr)
      return err(BFMRI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return BFMRI_OK;
}

}  // namespace

extern "C" {

size_t bfmri_pcg_static_capacity(void) { return kScratchBytes; }

size_t bfmri_pcg_static_bytes(size_t ld, int D) {
  if (ld < 1 || D < 1 || D > DMAX) return 0;
  const size_t lds = ld;
  const size_t rows = 4096;  // partial-sum rows: more than any cooperative grid can use
  return align256(sizeof(PcgCtrl)) + 256 + align256((rows * 8 + 8) * sizeof(double)) +
         align256((size_t)ntri(D) * lds * sizeof(double)) +
         5 * align256((size_t)D * lds * sizeof(double));
}

bfmri_status bfmri_pcg_solve_static(int N, int D, int neighbourhood, const int* nbr, size_t ld,
                                    const double* blocks, const double* scale, const double* b,
                                    double* x, double delta, int max_iter, void* cuda_stream,
                                    bfmri_solve_info* info) {
  if (N < 1 || D < 1 || D > DMAX) return err(BFMRI_ERR_INVALID_ARG, "need N >= 1 and 1 <= D <= 12");
  if (neighbourhood != 4 && neighbourhood != 6) return err(BFMRI_ERR_INVALID_ARG, "neighbourhood must be 4 or 6");
  if (ld < (size_t)N || ld % 32 != 0)
    return err(BFMRI_ERR_INVALID_ARG, "ld must be >= N and a multiple of 32");
  if (!nbr || !blocks || !scale || !b || !x) return err(BFMRI_ERR_INVALID_ARG, "NULL device pointer");
  if (!(delta > 0.0) || max_iter < 1) return err(BFMRI_ERR_INVALID_ARG, "need delta > 0 and max_iter >= 1");
  const size_t need = bfmri_pcg_static_bytes(ld, D);
  if (need > kScratchBytes)
    return err(BFMRI_ERR_INVALID_ARG, "problem needs " + std::to_string(need) +
                                          " bytes of scratch; the static area holds " +
                                          std::to_string(kScratchBytes) + " (reduce N or D)");
  void* base = nullptr;
  bfmri_status st = scratch_address(&base);
  if (st != BFMRI_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t lds = ld;   // scratch planes use the caller's leading dimension
  const size_t rows = 4096;
  unsigned char* p = static_cast<unsigned char*>(base);
  PcgCtrl* ctrl = reinterpret_cast<PcgCtrl*>(p);
  p += align256(sizeof(PcgCtrl));
  unsigned int* bar = reinterpret_cast<unsigned int*>(p);   // count, gen, err, bad voxel
  int* errw = reinterpret_cast<int*>(p + 8);
  int* bad = reinterpret_cast<int*>(p + 12);
  p += 256;
  double* part = reinterpret_cast<double*>(p);
  p += align256((rows * 8 + 8) * sizeof(double));
  double* mfac = reinterpret_cast<double*>(p);
  p += align256((size_t)ntri(D) * lds * sizeof(double));
  double* vec[5];
  for (int i = 0; i < 5; ++i) {
    vec[i] = reinterpret_cast<double*>(p);
    p += align256((size_t)D * lds * sizeof(double));
  }
  // state left by the previous call: clear what the solve needs to start at zero
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(PcgCtrl), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, 12, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0x7f, sizeof(int), s);
  if (e != cudaSuccess) return err(BFMRI_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  e = static_precond(D, N, ld, neighbourhood, nbr, blocks, scale, lds, mfac, bad, s);
  if (e != cudaSuccess) return err(BFMRI_ERR_CUDA, std::string("preconditioner: ") + cudaGetErrorString(e));
  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.N = N;
  a.ld = ld;
  a.ndir = neighbourhood;
  a.cw[0] = a.cw[1] = a.cw[2] = 1.0;   // the UGL prior
  a.nbr = nbr;
  a.blocks = blocks;
  a.mfac = nullptr;
  a.scale = scale;
  a.b = b;
  a.x = x;
  a.r = vec[0];
  a.u = vec[1];
  a.w = vec[2];
  a.p = vec[3];
  a.s = vec[4];
  a.part = part;
  a.part1 = part + rows * 4;
  a.bar.count = bar;
  a.bar.gen = bar + 1;
  a.bar.err = errw;
  a.bar.timeout_ns = 2000000000ull;
  a.ctrl = ctrl;
  a.delta = delta;
  a.max_iter = max_iter;
  a.skip_block = -1;
  a.max_grid = (int)rows;
  a.allow_resident = 1;
  a.mfac = mfac;
  int grid = 0;
  e = launch_pcg(D, a, s, &grid);
  if (e != cudaSuccess) return err(BFMRI_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  PcgCtrl c;
  int words[4];
  e = cudaMemcpyAsync(&c, ctrl, sizeof(c), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(words, bar, sizeof(words), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(BFMRI_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
  if (info) {
    info->iterations = c.iterations;
    info->refinements = c.restarts;
    info->rel_residual = c.rel_res;
    info->rel_residual0 = c.rel_res0;
  }
  if (words[2] == ERR_TIMEOUT_CODE) return err(BFMRI_ERR_TIMEOUT, "device grid barrier wait exceeded its time limit");
  if (words[3] != 0x7f7f7f7f)
    return err(BFMRI_ERR_NOT_SPD, "preconditioner block not positive definite at voxel " + std::to_string(words[3]));
  if (c.status == 4) return err(BFMRI_ERR_NOT_CONVERGED, "PCG reached max_iter");
  if (c.status == 3) return err(BFMRI_ERR_NOT_SPD, "PCG breakdown (p'Bp <= 0)");
  if (c.status == 7) return err(BFMRI_ERR_INVALID_ARG, "non-finite value in PCG");
  return BFMRI_OK;
}

}  // extern "C"
