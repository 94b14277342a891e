// Multi-right-hand-side PCG: S systems with one matrix B~ (probes, SVB samples) advance in
// lock-step inside one cooperative launch, each with its own CG scalars and stop test.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace bfmri {

// Per-RHS scalar state kept by the CTA that completes each reduction.
struct RhsState {
  double gam;      // r'M^-1 r of the previous iteration
  double alpha;    // current step
  double beta;     // current direction update
  double bb;       // ||b||^2
  double rr;       // latest ||r||^2
  double rr0;      // ||r||^2 of the start value
  int active;      // 1 while iterating
  int iters;       // iterations of the first (Lanczos-consistent) run
  int total;       // iterations including restarts
  int restarts;
  int hist_ok;     // 1 while no restart has happened (history is a Lanczos run)
  int status;      // 0 ok, 3 breakdown, 4 max_iter, 7 non-finite
};

// Operator and vectors of one right-hand side when the right-hand sides do not share a
// matrix (independent chains): packed blocks [ntri(D)][ld], block-Jacobi factor (or null),
// GMRF scales [D], b and x [D][ld]. With MrhsArgs.uneven the right-hand side also brings its
// own lattice (chains of different subjects, uneven masks): its voxels, neighbour
// directions, plane stride, neighbour planes [6][ld], red and black voxel lists and edge
// weights; otherwise those fields are unused and the launch's lattice applies.
struct MrhsRhsPtrs {
  const void* blocks;
  const void* mfac;
  const double* scale;
  const void* b;
  void* x;
  int N;
  int ndir;
  size_t ld;
  const int* nbr;
  const int* red;
  const int* black;
  int n_red;
  int n_black;
  double cw[3];
};

// Right-hand sides of one launch with uneven masks (MrhsArgs.uneven) at most.
constexpr int MRHS_UNEVEN_MAX_S = 128;

// Per right-hand side, accumulated over launches: iterations, solves, the first nonzero
// status (RhsState codes) and the relative residual of the last solve.
struct MrhsTally {
  long long iters;
  int solves;
  int status_any;
  double rel_res;
};

// Vector and operator arrays hold FP64 (f32 = 0) or FP32 (f32 = 1) elements; CG scalars,
// inner-product sums across threads and the stop test are FP64 in both cases.
struct MrhsArgs {
  int N;
  size_t ld;
  int ndir;
  int f32;
  const int* nbr;        // [6][ld]
  const void* blocks;    // [ntri(D)][ld]
  const void* mfac;      // [ntri(D)][ld] block-Jacobi factor (inverted diag) or null
  const double* scale;   // [D]
  int S;                 // number of right-hand sides
  size_t vs;             // stride between RHS (>= D * ld), in elements
  const void* b;         // [S] x [D][ld]
  void* x;               // [S] x [D][ld]: start values in, solutions out
  void* r;               // [S] x [D][ld] work
  void* u;
  void* w;
  void* p;
  void* s;
  double* part;          // [units][4]
  RhsState* st;          // [S]
  double* hist;          // [hist_len][S][2] CG (alpha, beta) of the first run, or null
  int hist_len;
  int* flags;            // [2]: any active, iteration counter
  GridBarrier bar;
  double delta;
  int max_iter;
  int max_restarts;
  int sm_cap;            // most SMs the grid may span (0 = all)
  const MrhsRhsPtrs* tab;  // [S] per-RHS operators, b and x (device), or null: all share
                           // blocks/mfac/scale and b, x are strided by vs
  MrhsTally* tally;      // [S] (device) or null
  // red-black symmetric SOR over the block-Jacobi blocks (plain solves only: the probes'
  // quadrature needs block-Jacobi): lattice colour lists shared by every right-hand side
  int ssor;
  double omega;
  const int* red;
  int n_red;
  const int* black;
  int n_black;
  // CG on the red-black reduced system instead (plain solves, FP64): needs mfac, the colour
  // lists and at most one (RHS, chunk) unit per warp (S <= warps of the grid)
  int reduced;
  double cw[3];          // edge weights of the x, y, z directions (1, 1, 1: UGL prior)
  // right-hand-side tile (FP32, one shared matrix, block-Jacobi or none, no SSOR, no
  // table): 2 or 4 = the vectors hold groups of `tile` right-hand sides interleaved per voxel
  // and component (element (i, k, n) at (i / tile) D ld tile + (k ld + n) tile + i % tile)
  // and k_mrhs_tile runs; 0 or 1 = the [S][D][ld] layout and k_mrhs
  int tile;
  // 1: every right-hand side has its own lattice in tab (which must be set), and the work
  // units are shared out in proportion to the right-hand sides' voxels (S <=
  // MRHS_UNEVEN_MAX_S; vs >= D ld of every right-hand side; N = the largest N)
  int uneven;
};

// Probe set-up and post-processing (log-determinant and trace probes).
struct ProbeArgs {
  int N;
  size_t ld;
  int ndir;
  int f32;              // b, x (and mfac for the right-hand sides) are FP32
  const int* nbr;
  const int* lin;
  const void* mfac;     // block-Jacobi factor (inverted diagonal), or null
  const double* mfac64; // FP64 factor for log det M
  int S;
  size_t vs;
  void* b;              // [S][D][ld]
  void* x;              // [S][D][ld]
  Rng rng;              // tag in c3's top byte; the probe index is the stream
  double cw[3];         // edge weights of the x, y, z directions
  int tile;             // layout of b and x: 2 or 4 = right-hand-side tiles (MrhsArgs.tile)
};
// what: 0 = probe right-hand sides b_i = L v_i and x_i = 0; 1 = per-voxel log det of the
// preconditioner into out[N]; 2 = trace partials into out[grid.x][S][D] (grid.x = ceil(N/128)).
cudaError_t launch_probe(int D, const ProbeArgs& a, int what, double* out, cudaStream_t s);
// out[c] = sum_g in[g * C + c] for c < C (fixed order per column).
cudaError_t launch_sum_columns(const double* in, int G, int C, double* out, cudaStream_t s);

// Launches the cooperative multi-RHS PCG for dimension D on `stream`.
cudaError_t launch_mrhs(int D, const MrhsArgs& a, cudaStream_t stream, int* units_out);
// Rows of the partial buffer the launch may need: S * chunks, bounded by this value.
int mrhs_max_units(int D, int S);

}  // namespace bfmri
