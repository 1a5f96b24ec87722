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
  int nface[3];               // interface faces of the stages of a step (slot of list_slot())
  int ncell[3];               // interface cells, by the same slots
  int nflip;                  // cells that changed material in the current step
  int err;                    // first latched m2c_status
  int pad0;
  long long err_cell;
  double t;
  long long step;
  long long stat_faces, stat_cells, stat_flips;
  double stat_dt;
  int pad[4];
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
  int riemann_fp32_start;
  // scheme options beyond the default (TVD RK2, modified van Albada, HLLC, CFL
  // time step): general = 1 when any differs, which selects the general
  // instantiation of the bulk kernel
  int general;
  int rk;             // Runge-Kutta order: 2 (TVD RK2), 3 (TVD RK3), 1 (forward Euler), Sec. 4.3
  int limiter;        // M2C_LIM_VAN_ALBADA or M2C_LIM_MC (App. D)
  int flux;           // M2C_FLUX_HLLC or M2C_FLUX_LLF (App. C)
  int pad2;
  double mc_alpha;    // alpha of the MC limiter
  double dt_fixed;    // > 0: constant time step instead of the CFL rule
  int geom;           // M2C_GEOM_CARTESIAN, _CYLINDRICAL or _SPHERICAL (Sec. 3.4): x is the radius
  int pad3;
  double x0;          // radius of the lower face of the first cell along x
  double band_beta, band_gamma;  // narrow-band level set: tube radii (lengths); gamma = 0: full domain
  double* W2;         // TVD RK3: the second stage state (workspace)
  double* phi2;
  // FIVER warm start: star pressure of each cell's x+, y+, z+ face from the face's
  // last exact Riemann solve (3 per cell; NaN: none); nullptr: no warm start
  double* pstar;
};

// Kernel modes: one Runge-Kutta stage each (the general bulk kernel only runs
// kStage2of3 and kStage3), or the residual alone.
//   kStage1     W1 = W + dt R(W)                                  (all schemes)
//   kStage2     W' = (W + (W1 + dt R(W1))) / 2                    (RK2, last)
//   kStage2of3  W2 = (3/4 W + 1/4 W1) + 1/4 dt R(W1)              (RK3)
//   kStage3     W' = (1/3 W + 2/3 W2) + 2/3 dt R(W2)              (RK3, last)
enum StageMode { kStage1 = 0, kStage2 = 1, kResidual = 2, kStage2of3 = 3, kStage3 = 4 };

// The state a stage reads (its own cell and the stencil), its work-list slot,
// and whether it is the last stage of a step (which writes the new state in
// place, detects flips and reduces the next time step).
__device__ __forceinline__ const double* stage_W(const Grid& g, int mode) {
  return (mode == kStage2 || mode == kStage2of3) ? g.W1 : (mode == kStage3 ? g.W2 : g.W);
}
__device__ __forceinline__ const double* stage_phi(const Grid& g, int mode) {
  return (mode == kStage2 || mode == kStage2of3) ? g.phi1 : (mode == kStage3 ? g.phi2 : g.phi);
}
__device__ __forceinline__ int list_slot(int mode) {
  return (mode == kStage2 || mode == kStage2of3) ? 1 : (mode == kStage3 ? 2 : 0);
}
__device__ __forceinline__ bool last_stage(int mode) { return mode == kStage2 || mode == kStage3; }

// Index of the cell whose state a ghost position i (outside [0, n)) takes:
// transmissive = the nearest cell (zero gradient), periodic = wrapped, symmetry =
// the mirror image across the side (its velocity component along the axis is
// negated by the caller, see mirrored()).
__device__ __forceinline__ int map_index(int i, int n, int lo_bc, int hi_bc) {
  if (i < 0) return lo_bc == M2C_BC_PERIODIC ? ((i % n) + n) % n : (lo_bc == M2C_BC_SYMMETRY ? -1 - i : 0);
  if (i >= n) return hi_bc == M2C_BC_PERIODIC ? i % n : (hi_bc == M2C_BC_SYMMETRY ? 2 * n - 1 - i : n - 1);
  return i;
}

// 1 when position i lies across a symmetry side of its axis.
__device__ __forceinline__ int mirrored(int i, int n, int lo_bc, int hi_bc) {
  return ((i < 0 && lo_bc == M2C_BC_SYMMETRY) || (i >= n && hi_bc == M2C_BC_SYMMETRY)) ? 1 : 0;
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

// Time step (Sec. 4.3): from the CFL number and the wave-speed maximum, or the
// grid's constant time step.
__device__ __forceinline__ double lam_to_dt(const Grid& g, unsigned long long bits) {
  if (g.dt_fixed > 0.0) return g.dt_fixed;
  double lam = __longlong_as_double((long long)bits);
  return g.cfl * g.h / lam;
}

}  // namespace m2c
