// Host/device interface of the persistent PCG solver for the block + stencil precision
//   B~ = blkdiag_n(B_n) + diag(s) (x) D        (paper Eq. wr full conditional; Section 3.1)
// over the in-mask voxel graph, in voxel-index structure-of-arrays layout: component k of
// voxel n of a vector lives at v[k * ld + n].
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace bfmri {

// Written by CTA 0 at the end of each solve. iter_total and status_any accumulate over
// solves until the host clears them.
struct PcgCtrl {
  int iterations;
  int restarts;       // FP64: true-residual restarts; mixed: outer refinement steps
  double rel_res;     // final true relative residual
  double rel_res0;    // relative residual of the start value
  int status;         // 0 ok, 3 breakdown (not SPD), 4 max_iter, 7 non-finite
  int status_any;     // first nonzero status since the last clear
  long long iter_total;
  long long solves;
};

struct PcgArgs {
  int N;
  size_t ld;             // plane stride (>= N, multiple of 32)
  int ndir;              // 4 or 6 neighbour planes used
  const int* nbr;        // [6][ld] compact neighbour index or -1 (-x,+x,-y,+y,-z,+z)
  const double* blocks;  // [ntri(D)][ld] data blocks (packed symmetric)
  const double* mfac;    // [ntri(D)][ld] preconditioner Cholesky factor (inverted diag) or null
  const double* scale;   // [D] prior scales (alpha or beta)
  const double* b;       // [D][ld] right-hand side
  double* x;             // [D][ld] start value in, solution out
  double* r;             // [D][ld] work (streaming variant)
  double* u;             // [D][ld] preconditioned residual, exchanged between CTAs
  double* w;             // [D][ld] work (streaming variant)
  double* p;
  double* s;
  double* part;          // [grid][4] reduction partials (even barrier generations)
  double* part1;         // [grid][4] reduction partials (odd barrier generations)
  GridBarrier bar;
  PcgCtrl* ctrl;
  double delta;          // stop when ||b - B x|| <= delta ||b|| (true residual, FP64)
  int max_iter;
  int skip_block;        // test hook (-1 off): this CTA never reaches the first barrier
  int max_grid;          // rows of the partial buffer: the launch never uses more CTAs
  int allow_resident;    // 1: use the register/shared-memory resident variant when N fits
  int sm_cap;            // most SMs the grid may span (0 = all)
  int res_per;           // resident variant: voxels per CTA (set by the launcher)
  // mixed precision: FP32 inner PCG inside FP64 iterative refinement
  int mixed;
  const float* blocks32; // [ntri(D)][ld] FP32 copies of blocks / mfac
  const float* mfac32;
  float* u32;            // [D][ld] inner preconditioned residual, exchanged between CTAs
  float* r32;            // [D][ld] streaming-variant work
  float* w32;
  float* p32;
  float* s32;
  float* d32;
  double inner_tol;      // relative tolerance of each inner solve
  int max_inner;         // inner iteration cap per refinement step
  // red-black symmetric SOR preconditioning (FP64 solvers only); mfac holds the
  // block-Jacobi factor of the diagonal blocks it is built on
  int ssor;
  double omega;          // relaxation, 0 < omega < 2
  const int* red;        // [n_red] compact indices of the voxels with x + y + z even
  int n_red;
  const int* black;      // [n_black] compact indices of the others
  int n_black;
  const unsigned char* colour;  // [ld] 0 red, 1 black (resident variant)
  // FP64 resident variant: CG on the red-black reduced system (Schur complement of the red
  // voxels) with the block factors mfac, equivalent to SSOR with omega = 1; the other
  // variants run that SSOR form instead (ssor = 1, omega = 1 must be set alongside)
  int reduced;
  double cw[3];          // edge weights of the x, y, z directions (1, 1, 1: UGL prior)
  int lanes;             // FP64 resident reduced solver (D <= 6): 1 = one lane per voxel
                         // (k_pcg_rbp), otherwise lane pairs (k_pcg_rbp2) when pair_slots is set
  int pair_per;          // the voxels per CTA that pair_slots was computed for
  int pair_slots;        // lane pairs per CTA: the most red, or black, voxels of any CTA
  // the L'L prior (D_w = L'L, L the weighted graph Laplacian): k_pcg_ltl, block-Jacobi or no
  // preconditioner, FP64 streaming; t is a [D][ld] plane for L v
  int ltl;
  double* t;
  // per-edge factors of C ([3][ld] BF16 of the edge from each voxel along +x, +y, +z, or
  // null): the FP64 streaming solver with block-Jacobi or no preconditioner only
  const unsigned short* ce;
  // anisotropic prior ([3][D] scale of direction d and component k, or null): the FP64
  // streaming solver with block-Jacobi or no preconditioner only; scale is then unused
  const double* scale3 = nullptr;
};

// Voxels per CTA of the resident solvers for N voxels on at most sm_cap SMs (0 = all): the
// grid spreads the voxels evenly, CTA b owning voxels [b per, (b + 1) per).
int resident_voxels_per_cta(int N, int sm_cap);

// Launches the cooperative persistent PCG kernel for dimension D (1..12) on `stream`.
// grid_out (may be null) receives the grid size used.
cudaError_t launch_pcg(int D, const PcgArgs& a, cudaStream_t stream, int* grid_out);

// Largest grid the cooperative launch of dimension D can use on the current device.
int pcg_max_grid(int D);

// One application of the solver's preconditioner, u = M^-1 r (a.r in, a.u out): block-Jacobi
// (mfac), none (mfac null), or red-black symmetric SOR (a.ssor) in its three colour phases
// as separate launches. Used to inspect the preconditioner; the solvers run the same
// per-voxel arithmetic inside their persistent launches.
cudaError_t launch_precond_apply(int D, const PcgArgs& a, cudaStream_t stream);

constexpr int PCG_THREADS = 256;
constexpr int DMAX = 12;

}  // namespace bfmri
