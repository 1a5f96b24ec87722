// Internal device structures of libm2cgpu: per-grid descriptors, the control
// block, the interface work lists and the launch helpers shared by the
// kernels and the C-ABI in m2c_solver.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "m2c_physics.cuh"

namespace m2c {

// One face between two cells of different material (its owner is the cell on
// the minus side; dir = 0, 1, 2 for x, y, z).
struct IfFace {
  long long cell;
  int dir;
  int pad;
};

// One cell with at least one interface face: its six face fluxes in the order
// x-, x+, y-, y+, z-, z+ (the bulk kernel writes the single-material faces, the
// FIVER kernel the interface faces).
struct IfCell {
  long long cell;
  double F[6][5];
};

// Control block of one grid, in the workspace.
struct Ctrl {
  unsigned long long lam[2];  // bit pattern of max_cells sum_d (|V_d| + c), by step parity
  int nface[2];               // interface faces of stage 1 / stage 2
  int ncell[2];               // interface cells of stage 1 / stage 2
  int nflip;                  // cells that changed material in the current step
  int err;                    // first latched m2c_status
  long long err_cell;
  double t;
  long long step;
  long long stat_faces, stat_cells, stat_flips;
  double stat_dt;
  int pad[6];
};

// Everything a kernel needs to know about one grid.
struct Grid {
  int nx, ny, nz, pad0;
  long long N;
  int bc[6];
  int active[3];    // axis has more than one cell
  int prec;         // m2c_precision
  double h, inv_h, cfl;
  EosDev eos[2];          // FP64 parameters (material 0: phi >= 0, 1: phi < 0)
  EosP<float> eosf[2];    // the same rounded once to FP32, for the mixed-precision kernels
  double* W;        // state W^n (caller's), updated in place by stage 2
  double* phi;      // level set (caller's)
  double* W1;       // stage-1 state
  double* phi1;
  double* phiC;     // reinitialisation scratch
  uint8_t* id;      // bit 0: material at the start of the step; bit 1: first-layer flag of the
                    // reinitialisation; bit 2: material at the end of the step
  int* cell_slot;   // interface-cell list slot of a cell (valid only for listed cells)
  IfFace* faces;
  IfCell* cells;
  long long* flips;
  int face_cap, cell_cap, flip_cap, pad1;
  Ctrl* ctrl;
  double* resR;     // residual outputs of m2c_residual
  double* resL;
  // tiling of the bulk stage kernel
  int tiles_x, tiles_y, tiles_z, tz;
  // reinitialisation after every reinit_every-th step (0: never), reinit_iters iterations
  int reinit_every, reinit_iters;
  // M2C_MIXED only: 1 = the FIVER Newton iteration starts on FP32 wave curves
  // and finishes with FP64 steps (riemann_solve_mixed); 0 = FP64 throughout
  int riemann_fp32_start, pad2;
};

enum StageMode { kStage1 = 0, kStage2 = 1, kResidual = 2 };

__device__ __forceinline__ int map_index(int i, int n, int lo_bc, int hi_bc) {
  if (i < 0) return lo_bc == M2C_BC_PERIODIC ? ((i % n) + n) % n : 0;
  if (i >= n) return hi_bc == M2C_BC_PERIODIC ? i % n : n - 1;
  return i;
}

__device__ __forceinline__ long long cell_of(const Grid& g, int i, int j, int k) {
  i = map_index(i, g.nx, g.bc[0], g.bc[1]);
  j = map_index(j, g.ny, g.bc[2], g.bc[3]);
  k = map_index(k, g.nz, g.bc[4], g.bc[5]);
  return ((long long)k * g.ny + j) * g.nx + i;
}

__device__ __forceinline__ void latch_error(Ctrl* c, int code, long long cell) {
  if (atomicCAS(&c->err, 0, code) == 0) c->err_cell = cell;
}

__device__ __forceinline__ double lam_to_dt(const Grid& g, unsigned long long bits) {
  double lam = __longlong_as_double((long long)bits);
  return g.cfl * g.h / lam;
}

}  // namespace m2c
