// Aggregation multigrid V-cycle as the PCG preconditioner of the W and A solves (a
// replacement of the paper's incomplete Cholesky, Section 3.1), FP64, any N.
//
// Level 0 is the voxel lattice; level l + 1 aggregates the voxels of level l in 2 x 2 x 2
// blocks (2 x 2 in-slice for the 4-neighbour prior). With piecewise-constant prolongation
// the Galerkin operator of every level has the form of B~: per-voxel blocks (the sums of the
// children's blocks) plus diag(scale) (x) a weighted graph Laplacian whose edge weights are
// the summed weights of the fine edges joining two aggregates. Smoothing: red-black block
// Gauss-Seidel (red then black before the coarse correction, black then red after it); the
// coarsest level takes a fixed number of symmetric red-black steps from zero. The cycle is
// symmetric positive definite.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "pcg.cuh"

namespace bfmri {

constexpr int MG_MAX_LEVELS = 4;

struct MgLevel {
  int N;
  size_t ld;
  const int* nbr;        // [6][ld] neighbour index per slot (-x,+x,-y,+y,-z,+z) or -1
  const double* wgt;     // [6][ld] edge weight of each slot (0 where there is no neighbour)
  const int* child;      // [8][ld] (levels >= 1) the aggregated voxels of the finer level, -1 padding
  const int* agg;        // [ld] (all but the coarsest) aggregate of each voxel on the next level
  const unsigned char* colour;   // [ld] 0 red (even coordinate sum), 1 black
  const int* red;        // the red voxels
  int n_red;
  const int* black;
  int n_black;
  const double* blocks;  // [ntri(D)][ld] per-voxel blocks (level 0: the system's data blocks)
  double* fac;           // [ntri(D)][ld] Cholesky factor (inverted diagonal) of blocks + diag(scale) deg
  double* b;             // [D][ld] right-hand side of the level (level 0: the PCG residual)
  double* x;             // [D][ld] the level's correction (level 0: the preconditioned residual)
  double* r;             // [D][ld] the level's residual b - A x
};

struct MgArgs {
  int L;                 // levels (>= 1)
  int coarse_steps;      // symmetric Gauss-Seidel steps on the coarsest level
  MgLevel lv[MG_MAX_LEVELS];
  const double* scale;   // [D] prior scales (alpha or beta)
  const double* b;       // [D][ld0] right-hand side of the solve
  double* x;             // [D][ld0] start value in, solution out
  double* r;             // [D][ld0] PCG residual (= level 0's b)
  double* z;             // [D][ld0] preconditioned residual (= level 0's x)
  double* p;
  double* q;
  double* part;          // [grid][4] reduction rows (even barrier generations)
  double* part1;         // [grid][4] (odd generations)
  int max_grid;
  int sm_cap;            // most SMs the grid may span (0 = all)
  GridBarrier bar;
  PcgCtrl* ctrl;
  double delta;
  int max_iter;
  int* bad_voxel;        // smallest voxel index whose coarse block is not positive definite
  int apply_only;        // 1: z = M^-1 r once (inspection), no solve
};

// Coarse blocks (sums of the children's) and the Gauss-Seidel factors of levels 1..L-1.
cudaError_t launch_mg_setup(int D, const MgArgs& a, cudaStream_t stream);
// The whole PCG solve with the V-cycle preconditioner in one cooperative launch (or, with
// apply_only, one application of the V-cycle to r).
cudaError_t launch_pcg_mg(int D, const MgArgs& a, cudaStream_t stream, int* grid_out);
// Largest grid of launch_pcg_mg on the current device.
int pcg_mg_max_grid(int D);

}  // namespace bfmri
