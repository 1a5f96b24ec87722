// libm2cgpu: GB300 (sm_103a) kernels and C-ABI of the multi-material
// finite-volume step of M2C (arXiv 2508.16387), declared in include/m2c.h.
//
// One time step (Sec. 2.3 steps (1)-(6), RK2 of Sec. 4.3) is eight launches:
//   stage 1: k_stage (bulk) -> k_fiver (interface faces) -> k_finish (interface cells)
//   stage 2: k_stage        -> k_fiver                  -> k_finish
//   [k_reinit x iterations, every reinit_every steps] -> k_phase_fix -> k_end_step
// The bulk kernel marches a 32 x TY column tile along z: a plane of primitive
// states with a two-cell halo in shared memory, a register window of planes
// along z, MUSCL face states and HLLC fluxes per face computed once, the
// residual sum, the level-set residual and the Runge-Kutta update fused in
// the same pass. Faces whose two cells have different materials are not
// solved there: they are compacted by warp ballot into a work list and solved
// packed by k_fiver (exact Riemann problem, FP64), and the cells touching them
// are finished by k_finish. The time step is reduced on the device (max of
// the wave-speed sum, atomically, in the kernels that write the new state).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "m2c_kernels.cuh"
#include "m2c_device.cuh"
#include "m2c_riemann.cuh"
#include "m2c_stage.h"

namespace m2c {

// ---------------------------------------------------------------------------
// FIVER on the packed interface faces (Sec. 4.2): exact two-material Riemann
// problem on the normal projections of the two cell states (their face states
// are the cell states, Reading R11), star states with each side's tangential
// velocity (Reading R8), F_ij = Phi(W_ij, W*_ij; EOS_i) and
// F_ji = Phi(W*_ji, W_ji; EOS_j) (Reading R16), FP64.
// ---------------------------------------------------------------------------

template <int D, typename R>
__device__ __forceinline__ void fiver_fluxes(const FaceState<R>& A, const FaceState<R>& SA, const FaceState<R>& SB,
                                             const FaceState<R>& B, R Fa[5], R Fb[5], int flux) {
  if (flux == M2C_FLUX_LLF) {
    llf<D, R>(A, SA, Fa);
    llf<D, R>(SB, B, Fb);
    return;
  }
  hllc<D, R>(A, SA, Fa);
  hllc<D, R>(SB, B, Fb);
}

// The two fluxes of an interface face from its cell states (Pa, Pb) and star
// states (Sa, Sb), in the working precision R of the grid's fluxes: FP64, or
// FP32 on the mixed path (as the bulk kernel's HLLC); false if a face state is
// not admissible.
template <typename R>
__device__ __forceinline__ bool fiver_face_fluxes(const EosP<R>& qa, const EosP<R>& qb, const double Pa[5],
                                                  const double Sa[5], const double Sb[5], const double Pb[5], int d,
                                                  int flux, double Fa[5], double Fb[5]) {
  FaceState<R> A, SA, SB, B;
  bool ok = make_face<R, true>(qa, to_r<R>(Pa[0]), to_r<R>(Pa[1]), to_r<R>(Pa[2]), to_r<R>(Pa[3]), to_r<R>(Pa[4]), A);
  ok = make_face<R, true>(qa, to_r<R>(Sa[0]), to_r<R>(Sa[1]), to_r<R>(Sa[2]), to_r<R>(Sa[3]), to_r<R>(Sa[4]), SA) && ok;
  ok = make_face<R, true>(qb, to_r<R>(Sb[0]), to_r<R>(Sb[1]), to_r<R>(Sb[2]), to_r<R>(Sb[3]), to_r<R>(Sb[4]), SB) && ok;
  ok = make_face<R, true>(qb, to_r<R>(Pb[0]), to_r<R>(Pb[1]), to_r<R>(Pb[2]), to_r<R>(Pb[3]), to_r<R>(Pb[4]), B) && ok;
  R fa[5], fb[5];
  if (d == 0) fiver_fluxes<0, R>(A, SA, SB, B, fa, fb, flux);
  else if (d == 1) fiver_fluxes<1, R>(A, SA, SB, B, fa, fb, flux);
  else fiver_fluxes<2, R>(A, SA, SB, B, fa, fb, flux);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Fa[v] = to_d<R>(fa[v]);
    Fb[v] = to_d<R>(fb[v]);
  }
  return ok;
}

// One warp-sized block per 32 faces, so that the few warps of a typical
// interface spread evenly over the SMs (each is FP64-pipe bound).
constexpr int kFiverThreads = 32;
__global__ void __launch_bounds__(kFiverThreads, 1) k_fiver(const Grid* __restrict__ grids, int mode) {
  const Grid& G = grids[blockIdx.y];
  Ctrl* ctrl = G.ctrl;
  const int slot = list_slot(mode);
  const int n = min(ctrl->nface[slot], G.face_cap);
  const double* __restrict__ Ws = stage_W(G, mode);
  const long long N = G.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const IfFace f = G.faces[i];
    const long long ca = f.cell;
    const int ix = (int)(ca % G.nx), iy = (int)((ca / G.nx) % G.ny), iz = (int)(ca / ((long long)G.nx * G.ny));
    const int d = f.dir;
    const long long cb = cell_of(G, ix + (d == 0), iy + (d == 1), iz + (d == 2));
    const int ia = G.id[ca] & 1, ib = G.id[cb] & 1;
    const EosDev& qa = G.eos[ia];
    const EosDev& qb = G.eos[ib];
    double Pa[5], Pb[5];
    bool ok = cons_to_prim<double, true>(qa, qa, Ws, N, ca, Pa);
    ok = cons_to_prim<double, true>(qb, qb, Ws, N, cb, Pb) && ok;
    double Fa[5] = {0, 0, 0, 0, 0}, Fb[5] = {0, 0, 0, 0, 0};
    RiemannOut rs;
    int its = 0;
    int st = M2C_ENONPHYS;
    // Newton starts from this face's star pressure of its last solve (the previous
    // stage), else from the PVRS estimate; the residual alone (kResidual) always
    // starts from PVRS
    double* pst = (mode != kResidual && G.pstar) ? G.pstar + 3 * ca + d : nullptr;
    const double p_start = pst ? *pst : (double)NAN;
    if (ok) {
      // material 0 is put on the left of the 1D problem (the mirror image, normal
      // velocities negated, when it is on the plus side), so that every lane of a
      // warp evaluates the same wave curves; the mirrored solve is the same
      // arithmetic with the two sides exchanged (sums commute exactly), and its
      // solution is mirrored back below
      const bool mirror = ia > ib;
      const EosDev& q0 = mirror ? qb : qa;
      const EosDev& q1 = mirror ? qa : qb;
      const double* P0 = mirror ? Pb : Pa;
      const double* P1 = mirror ? Pa : Pb;
      const double sgn = mirror ? -1.0 : 1.0;
      if (G.prec == M2C_MIXED && G.riemann_fp32_start)
        st = riemann_solve_mixed(G.eosf[mirror ? ib : ia], q0, P0[0], sgn * P0[1 + d], P0[4], G.eosf[mirror ? ia : ib], q1,
                                 P1[0], sgn * P1[1 + d], P1[4], rs, its, p_start);
      else
        st = riemann_solve(q0, P0[0], sgn * P0[1 + d], P0[4], q1, P1[0], sgn * P1[1 + d], P1[4], rs, its, p_start);
      if (pst && st == M2C_OK) *pst = rs.p;
      if (mirror) {
        const double r = rs.rhoL;
        rs.rhoL = rs.rhoR;
        rs.rhoR = r;
        rs.u = -rs.u;
      }
    }
    if (st == M2C_OK) {
      double Sa[5] = {rs.rhoL, Pa[1], Pa[2], Pa[3], rs.p};
      double Sb[5] = {rs.rhoR, Pb[1], Pb[2], Pb[3], rs.p};
      Sa[1 + d] = rs.u;
      Sb[1 + d] = rs.u;
      const bool okf = G.prec == M2C_MIXED
                           ? fiver_face_fluxes<float>(G.eosf[ia], G.eosf[ib], Pa, Sa, Sb, Pb, d, G.flux, Fa, Fb)
                           : fiver_face_fluxes<double>(qa, qb, Pa, Sa, Sb, Pb, d, G.flux, Fa, Fb);
      if (!okf) st = M2C_ENONPHYS;
    }
    if (st != M2C_OK) {
      latch_error(ctrl, st, ca);
#pragma unroll
      for (int v = 0; v < 5; ++v) Fa[v] = Fb[v] = 0.0;
    }
    // a slot is trusted only if it is inside this stage's list and points back
    // at the cell (an overflowed list leaves slots unwritten; the error is latched)
    const int ncl = min(ctrl->ncell[slot], G.cell_cap);
    const int sa = G.cell_slot[ca], sb = G.cell_slot[cb];
    const bool oka = sa >= 0 && sa < ncl && G.cells[sa].cell == ca;
    const bool okb = sb >= 0 && sb < ncl && G.cells[sb].cell == cb;
    if (!oka || !okb) latch_error(ctrl, M2C_EOVERFLOW, ca);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      if (oka) G.cells[sa].F[2 * d + 1][v] = Fa[v];
      if (okb) G.cells[sb].F[2 * d][v] = Fb[v];
    }
  }
}

// Interface cells: residual from the six stored face fluxes in the fixed
// association ((x) + (y)) + (z), then the stage update of the mode (the same
// formulas as the bulk kernel's).
__global__ void __launch_bounds__(128) k_finish(const Grid* __restrict__ grids, int mode) {
  __shared__ double s_red[32];
  const Grid& G = grids[blockIdx.y];
  Ctrl* ctrl = G.ctrl;
  const int slot = list_slot(mode);
  const int n = min(ctrl->ncell[slot], G.cell_cap);
  const long long N = G.N;
  const long long step = ctrl->step;
  const double dt = mode == kResidual ? 0.0 : lam_to_dt(G, ctrl->lam[step & 1]);
  const double ih = G.inv_h;
  double lam_max = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const IfCell& e = G.cells[i];
    const long long c = e.cell;
    double res[5];
#pragma unroll
    for (int v = 0; v < 5; ++v)
      res[v] = ((e.F[0][v] - e.F[1][v]) * ih + (e.F[2][v] - e.F[3][v]) * ih) + (e.F[4][v] - e.F[5][v]) * ih;
    if (G.geom != M2C_GEOM_CARTESIAN) {
      // spherical / cylindrical source term (Sec. 3.4), FP64, as in the bulk kernel
      const double* __restrict__ Ws = stage_W(G, mode);
      const int m = G.id[c] & 1;
      double P[5];
      if (!cons_to_prim<double, true>(G.eos[m], G.eos[m], Ws, N, c, P)) latch_error(ctrl, M2C_ENONPHYS, c);
      const double r = G.x0 + ((double)(c % G.nx) + 0.5) * G.h;
      const double a = (G.geom == M2C_GEOM_SPHERICAL ? 2.0 : 1.0) / r * P[1];
#pragma unroll
      for (int v = 0; v < 4; ++v) res[v] = res[v] - a * Ws[v * N + c];
      res[4] = res[4] - a * (Ws[4 * N + c] + P[4]);
    }
    if (mode == kResidual) {
#pragma unroll
      for (int v = 0; v < 5; ++v) G.resR[v * N + c] = res[v];
    } else if (mode == kStage1) {
#pragma unroll
      for (int v = 0; v < 5; ++v) G.W1[v * N + c] = G.W[v * N + c] + dt * res[v];
    } else if (mode == kStage2of3) {
#pragma unroll
      for (int v = 0; v < 5; ++v)
        G.W2[v * N + c] = (0.75 * G.W[v * N + c] + 0.25 * G.W1[v * N + c]) + 0.25 * dt * res[v];
    } else {
      if (mode == kStage3) {
#pragma unroll
        for (int v = 0; v < 5; ++v)
          G.W[v * N + c] = (G.W[v * N + c] / 3.0 + 2.0 / 3.0 * G.W2[v * N + c]) + 2.0 / 3.0 * dt * res[v];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) G.W[v * N + c] = 0.5 * (G.W[v * N + c] + (G.W1[v * N + c] + dt * res[v]));
      }
      const int id0 = G.id[c] & 1;
      const bool flip = lt0(G.phi[c]) != (id0 == 1);
      if (!flip) {
        bool ok;
        const double lam = wave_sum(G, id0, G.W, N, c, ok);
        if (!ok) latch_error(ctrl, M2C_ENONPHYS, c);
        lam_max = fmax(lam_max, lam);
      }
    }
  }
  if (last_stage(mode)) block_max_to(lam_max, &ctrl->lam[(step + 1) & 1], s_red);
}

// Forward Euler (Sec. 4.3): the one stage wrote W1 = W + dt R(W); the step
// takes it as the new state, detects the cells whose level set changed sign
// and reduces the next time step, as the last stage of the other schemes does.
__global__ void __launch_bounds__(256) k_commit_euler(const Grid* __restrict__ grids) {
  __shared__ double s_red[32];
  const Grid& G = grids[blockIdx.y];
  Ctrl* ctrl = G.ctrl;
  const long long N = G.N;
  double lam_max = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int v = 0; v < 5; ++v) G.W[v * N + c] = G.W1[v * N + c];
    const double pn = G.phi1[c];
    G.phi[c] = pn;
    const int id0 = G.id[c] & 1;
    const bool neg = lt0(pn);
    G.id[c] = (uint8_t)(id0 | (neg ? 4 : 0));
    if (neg != (id0 == 1)) {
      const int s = atomicAdd(&ctrl->nflip, 1);
      if (s < G.flip_cap) G.flips[s] = c;
      else latch_error(ctrl, M2C_EOVERFLOW, c);
    } else {
      bool ok;
      const double lam = wave_sum(G, id0, G.W, N, c, ok);
      if (!ok) latch_error(ctrl, M2C_ENONPHYS, c);
      lam_max = fmax(lam_max, lam);
    }
  }
  block_max_to(lam_max, &ctrl->lam[(ctrl->step + 1) & 1], s_red);
}

// ---------------------------------------------------------------------------
// Reinitialisation (Eq. reinit, Sec. 4.4): one Jacobi iteration
// phi' = phi - dtau S(phi0) (G(phi) - 1), Godunov upwind |grad phi|,
// S = phi0/sqrt(phi0^2 + h^2), dtau = h/2, first-layer cells fixed. phi stays
// FP64 in memory; the update is computed in R (FP32 on the mixed path: the
// level set is a distance to within the grid's resolution, far above FP32
// rounding).
// ---------------------------------------------------------------------------
constexpr int kReinitChunk = 32;  // planes marched by one thread
template <typename R>
__global__ void __launch_bounds__(256) k_reinit(const Grid* __restrict__ grids, int it) {
  const Grid& G = grids[blockIdx.y];
  // each grid follows its own schedule: after its steps reinit_every, 2 reinit_every, ...
  const int nits = G.reinit_iters;
  if (G.reinit_every <= 0 || it > nits || (G.ctrl->step + 1) % G.reinit_every != 0) return;
  // phi0 is the state phi; iterations alternate phi1 and phiC and the last one
  // writes phi (a single iteration ends in phi1 and is copied back)
  const double* __restrict__ src = it == 1 ? G.phi : ((it % 2 == 0) ? G.phi1 : G.phiC);
  double* __restrict__ dst = (it == nits && it > 1) ? G.phi : ((it % 2 == 1) ? G.phi1 : G.phiC);
  const bool first_iter = it == 1;  // src is phi0: the first-layer flags are set from it
  const double* phi0 = G.phi;  // also dst in the last of several iterations (read first, same cell)
  uint8_t* __restrict__ idg = G.id;
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const unsigned ncol = (unsigned)nx * (unsigned)ny;
  const long long nxy = ncol;
  const unsigned nchunk = (unsigned)((nz + kReinitChunk - 1) / kReinitChunk);
  const R h = (R)G.h, ih = (R)G.inv_h, dtau = (R)(0.5 * G.h);
  // one thread marches one column (i, j) over a chunk of planes with a
  // three-plane window of src in registers; x and y neighbours are loaded
  for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w < ncol * nchunk; w += gridDim.x * blockDim.x) {
    const unsigned chunk = w / ncol, col = w - chunk * ncol;
    const int j = (int)(col / (unsigned)nx), i = (int)(col - (unsigned)j * (unsigned)nx);
    const int k0 = (int)chunk * kReinitChunk, k1 = min(k0 + kReinitChunk, nz);
    const long long oxm = (long long)j * nx + map_index(i - 1, nx, G.bc[0], G.bc[1]);
    const long long oxp = (long long)j * nx + map_index(i + 1, nx, G.bc[0], G.bc[1]);
    const long long oym = (long long)map_index(j - 1, ny, G.bc[2], G.bc[3]) * nx + i;
    const long long oyp = (long long)map_index(j + 1, ny, G.bc[2], G.bc[3]) * nx + i;
    double sm = src[map_index(k0 - 1, nz, G.bc[4], G.bc[5]) * nxy + col];
    double s0 = src[k0 * nxy + col];
    for (int k = k0; k < k1; ++k) {
      const long long base = k * nxy, c = base + col;
      const double sp = src[map_index(k + 1, nz, G.bc[4], G.bc[5]) * nxy + col];
      const double nbv[6] = {src[base + oxm], src[base + oxp], src[base + oym], src[base + oyp], sm, sp};
      const double p0 = first_iter ? s0 : phi0[c];
      bool first;
      if (first_iter) {
        const bool neg0 = lt0(p0);
        first = false;
#pragma unroll
        for (int q = 0; q < 6; ++q) first = first || (lt0(nbv[q]) != neg0);
        idg[c] = (uint8_t)((idg[c] & 5) | (first ? 2 : 0));
      } else {
        first = (idg[c] & 2) != 0;
      }
      if (first) {
        dst[c] = s0;
      } else {
        const R cr = to_r<R>(s0);
        R G2[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const R a = (cr - to_r<R>(nbv[2 * d])) * ih;
          const R b = (to_r<R>(nbv[2 * d + 1]) - cr) * ih;
          R x, y;
          if (!lt0(p0)) {
            x = fmax(a, (R)0);
            y = fmin(b, (R)0);
          } else {
            x = fmin(a, (R)0);
            y = fmax(b, (R)0);
          }
          G2[d] = fmax(x * x, y * y);
        }
        const R Gn = sqrt((G2[0] + G2[1]) + G2[2]);
        const R pr = to_r<R>(p0);
        const R S = pr / sqrt(pr * pr + h * h);
        if constexpr (sizeof(R) == 8) dst[c] = s0 - dtau * S * (Gn - (R)1);
        else dst[c] = s0 - f2d(dtau * S * (Gn - (R)1));
      }
      sm = s0;
      s0 = sp;
    }
  }
}

__global__ void k_copy_phi1(const Grid* __restrict__ grids) {
  const Grid& G = grids[blockIdx.y];
  if (G.reinit_every <= 0 || G.reinit_iters != 1 || (G.ctrl->step + 1) % G.reinit_every != 0) return;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < G.N; c += (long long)gridDim.x * blockDim.x)
    G.phi[c] = G.phi1[c];
}

// Narrow band (Sec. 4.4): after the Runge-Kutta update and the scheduled
// reinitialisation the level set is clipped to [-gamma, gamma] (a plateau
// beyond the tube; the signs, hence the materials, are unchanged).
__global__ void __launch_bounds__(256) k_band_clip(const Grid* __restrict__ grids) {
  const Grid& G = grids[blockIdx.y];
  if (!(G.band_gamma > 0.0)) return;
  const double gam = G.band_gamma;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < G.N; c += (long long)gridDim.x * blockDim.x)
    G.phi[c] = fmax(-gam, fmin(gam, G.phi[c]));
}

// ---------------------------------------------------------------------------
// Phase update (Sec. 2.3 step (6)): a cell whose material changed takes the
// mean primitive state of its face neighbours that were and are of its new
// material, else of its 26-neighbourhood, converted with the new EOS. With no
// such neighbour at all (a fragment smaller than a cell) the cell keeps its
// material and state, and its level set takes that material's sign.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_phase_fix(const Grid* __restrict__ grids) {
  __shared__ double s_red[32];
  const Grid& G = grids[blockIdx.y];
  Ctrl* ctrl = G.ctrl;
  const int n = min(ctrl->nflip, G.flip_cap);
  const long long N = G.N;
  double lam_max = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const long long c = G.flips[t];
    const int i = (int)(c % G.nx), j = (int)((c / G.nx) % G.ny), k = (int)(c / ((long long)G.nx * G.ny));
    const int m = (G.id[c] >> 2) & 1;  // material at the end of the step
    const EosDev& q = G.eos[m];
    double sum[5] = {0, 0, 0, 0, 0};
    int cnt = 0;
    // a neighbour position across a symmetry side is the mirror image of a cell
    // inside, its velocity component along that axis negated
    auto take = [&](int ii, int jj, int kk) {
      const long long nb = cell_of(G, ii, jj, kk);
      const int old_id = G.id[nb] & 1;
      const int new_id = (G.id[nb] >> 2) & 1;
      if (old_id == m && new_id == m) {
        double P[5];
        if (!cons_to_prim<double, true>(q, q, G.W, N, nb, P)) latch_error(ctrl, M2C_ENONPHYS, nb);
        if (mirrored(ii, G.nx, G.bc[0], G.bc[1])) P[1] = -P[1];
        if (mirrored(jj, G.ny, G.bc[2], G.bc[3])) P[2] = -P[2];
        if (mirrored(kk, G.nz, G.bc[4], G.bc[5])) P[3] = -P[3];
#pragma unroll
        for (int v = 0; v < 5; ++v) sum[v] = sum[v] + P[v];
        ++cnt;
      }
    };
    take(i - 1, j, k);
    take(i + 1, j, k);
    take(i, j - 1, k);
    take(i, j + 1, k);
    take(i, j, k - 1);
    take(i, j, k + 1);
    if (cnt == 0) {
      for (int dk = -1; dk <= 1; ++dk)
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di)
            if (di || dj || dk) take(i + di, j + dj, k + dk);
    }
    if (cnt == 0) {
      const int old_id = 1 - m;
      const double pv = G.phi[c];
      G.phi[c] = old_id ? -fmax(fabs(pv), 1e-12 * G.h) : fabs(pv);
      bool ok;
      const double lam = wave_sum(G, old_id, G.W, N, c, ok);
      if (!ok) latch_error(ctrl, M2C_ENONPHYS, c);
      lam_max = fmax(lam_max, lam);
      continue;
    }
    double P[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) P[v] = sum[v] / cnt;
    double e, c2;
    if (!eos_e_c2<double, true>(q, P[0], 1.0 / P[0], P[4], e, c2)) latch_error(ctrl, M2C_ENONPHYS, c);
    G.W[c] = P[0];
    G.W[N + c] = P[0] * P[1];
    G.W[2 * N + c] = P[0] * P[2];
    G.W[3 * N + c] = P[0] * P[3];
    G.W[4 * N + c] = P[0] * e + 0.5 * P[0] * ((P[1] * P[1] + P[2] * P[2]) + P[3] * P[3]);
    bool ok;
    const double lam = wave_sum(G, m, G.W, N, c, ok);
    lam_max = fmax(lam_max, lam);
  }
  block_max_to(lam_max, &ctrl->lam[(ctrl->step + 1) & 1], s_red);
}

// End of a step: advance t and the step counter, keep the counters of the
// step for m2c_get_stats and reset the work lists for the next step.
__global__ void k_end_step(const Grid* __restrict__ grids, int ngrid) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= ngrid) return;
  const Grid& G = grids[gi];
  Ctrl* c = G.ctrl;
  const long long s = c->step;
  const double dt = lam_to_dt(G, c->lam[s & 1]);
  c->t = c->t + dt;
  c->stat_faces = c->nface[0];
  c->stat_cells = c->ncell[0];
  c->stat_flips = c->nflip;
  c->nface[0] = c->nface[1] = c->nface[2] = 0;
  c->ncell[0] = c->ncell[1] = c->ncell[2] = 0;
  c->nflip = 0;
  c->lam[s & 1] = 0ull;  // slot of step s + 2
  c->step = s + 1;
  c->stat_dt = lam_to_dt(G, c->lam[(s + 1) & 1]);
}

// Wave-speed maximum of the current state (first time step).
__global__ void __launch_bounds__(256) k_lam_init(const Grid* __restrict__ grids) {
  __shared__ double s_red[32];
  const Grid& G = grids[blockIdx.y];
  double lam_max = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < G.N; c += (long long)gridDim.x * blockDim.x) {
    const int m = lt0(G.phi[c]) ? 1 : 0;
    bool ok;
    const double lam = wave_sum(G, m, G.W, G.N, c, ok);
    if (!ok) latch_error(G.ctrl, M2C_ENONPHYS, c);
    lam_max = fmax(lam_max, lam);
  }
  block_max_to(lam_max, &G.ctrl->lam[G.ctrl->step & 1], s_red);
}

// Primitive fields (rho, u, v, w, p) of the current state, FP64, with the EOS
// of each cell's material (Sec. 3.3); the inverse of k_prims_to_state.
__global__ void k_state_to_prims(const Grid* __restrict__ grids, double* __restrict__ prims) {
  const Grid& G = grids[0];
  const long long N = G.N;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const int m = lt0(G.phi[c]) ? 1 : 0;
    double P[5];
    if (!cons_to_prim<double, true>(G.eos[m], G.eos[m], G.W, N, c, P)) latch_error(G.ctrl, M2C_ENONPHYS, c);
#pragma unroll
    for (int v = 0; v < 5; ++v) prims[v * N + c] = P[v];
  }
}

__global__ void k_prims_to_state(const Grid* __restrict__ grids, const double* __restrict__ prims) {
  const Grid& G = grids[0];
  const long long N = G.N;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const int m = lt0(G.phi[c]) ? 1 : 0;
    const double rho = prims[c], u = prims[N + c], v = prims[2 * N + c], w = prims[3 * N + c], p = prims[4 * N + c];
    double e, c2;
    if (!eos_e_c2<double, true>(G.eos[m], rho, 1.0 / rho, p, e, c2)) latch_error(G.ctrl, M2C_ENONPHYS, c);
    G.W[c] = rho;
    G.W[N + c] = rho * u;
    G.W[2 * N + c] = rho * v;
    G.W[3 * N + c] = rho * w;
    G.W[4 * N + c] = rho * e + 0.5 * rho * ((u * u + v * v) + w * w);
  }
}

__global__ void k_riemann_batch(int n, EosDev qL, const double* __restrict__ L, EosDev qR,
                                const double* __restrict__ Rr, double* __restrict__ out, int* __restrict__ iters,
                                int* __restrict__ status, int mixed, EosP<float> qLf, EosP<float> qRf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    RiemannOut o;
    int its = 0;
    const int st =
        mixed ? riemann_solve_mixed(qLf, qL, L[i], L[n + i], L[2 * n + i], qRf, qR, Rr[i], Rr[n + i], Rr[2 * n + i], o,
                                    its)
              : riemann_solve(qL, L[i], L[n + i], L[2 * n + i], qR, Rr[i], Rr[n + i], Rr[2 * n + i], o, its);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    out[i] = st ? nan : o.p;
    out[n + i] = st ? nan : o.u;
    out[2 * n + i] = st ? nan : o.rhoL;
    out[3 * n + i] = st ? nan : o.rhoR;
    if (iters) iters[i] = its;
    if (status) status[i] = st;
  }
}

// Post-shock state from the right-facing wave curve of the Riemann solver.
__global__ void k_shock_state(EosDev q, double rho, double u, double p, double p1, double* out, int* status) {
  Side K;
  if (!make_side(q, rho, u, p, K) || !(p1 > p)) {
    *status = M2C_EINVAL;
    return;
  }
  double f, df, rs;
  const int st = wave(q, K, p1, f, df, rs);
  *status = st;
  if (st) return;
  out[0] = rs;
  out[1] = K.u + f;
  out[2] = (rs * out[1] - K.rho * K.u) / (rs - K.rho);
}

}  // namespace m2c

// ===========================================================================
// C-ABI
// ===========================================================================
using namespace m2c;

struct m2c_ctx {
  Grid host;            // host copy of the device descriptor
  Grid* dev_grid;       // in the workspace
  long long* dev_tiles; // tile_begin[2] in the workspace
  cudaStream_t stream;
  int ty;               // tile rows of the bulk kernel
  int reinit_every, reinit_iters;
  long long host_step;
  bool has_state, eos_set[2], dirty, lam_valid;
  bool profiling, profile_bulk_only;
  size_t ws_bytes;      // size of the caller's workspace
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;  // event pairs around launches while profiling
  std::vector<int> ev_kind;
  size_t ev_used;
  // m2c_step_host: the upload stream, one event per state component for the end
  // of its download and of its upload, and the host arrays of the last call
  cudaStream_t copy_in = nullptr;
  cudaEvent_t down_ev[6] = {}, up_ev[6] = {};
  const double* last_W_host = nullptr;
  const double* last_phi_host = nullptr;
  std::string err;
};

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t grid, tiles, ctrl, W1, phi1, phiC, id, slot, faces, cells, flips, pstar, W2, phi2, total;
  int face_cap, cell_cap, flip_cap;
};

// rk = 3 appends the second stage state of TVD RK3 (W2, phi2) to the layout of
// the other schemes, which stays a prefix.
Layout layout_for(long long N, int rk = 2) {
  Layout L{};
  L.face_cap = (int)std::min<long long>(std::max<long long>(4096, N / 4), 1ll << 30);
  L.cell_cap = (int)std::min<long long>(std::max<long long>(2048, N / 8), 1ll << 30);
  L.flip_cap = (int)std::min<long long>(std::max<long long>(1024, N / 16), 1ll << 30);
  size_t o = 0;
  L.grid = o; o = align_up(o + sizeof(Grid));
  L.tiles = o; o = align_up(o + 2 * sizeof(long long));
  L.ctrl = o; o = align_up(o + sizeof(Ctrl));
  L.W1 = o; o = align_up(o + sizeof(double) * 5 * N);
  L.phi1 = o; o = align_up(o + sizeof(double) * N);
  L.phiC = o; o = align_up(o + sizeof(double) * N);
  L.id = o; o = align_up(o + N);
  L.slot = o; o = align_up(o + sizeof(int) * N);
  L.faces = o; o = align_up(o + sizeof(IfFace) * (size_t)L.face_cap);
  L.cells = o; o = align_up(o + sizeof(IfCell) * (size_t)L.cell_cap);
  L.flips = o; o = align_up(o + sizeof(long long) * (size_t)L.flip_cap);
  L.pstar = o; o = align_up(o + sizeof(double) * 3 * N);
  L.W2 = L.phi2 = 0;
  if (rk == 3) {
    L.W2 = o; o = align_up(o + sizeof(double) * 5 * N);
    L.phi2 = o; o = align_up(o + sizeof(double) * N);
  }
  L.total = o;
  return L;
}

// Error text of the calls that take no context (m2c_last_error(NULL)).
thread_local std::string g_noctx_error;

// set_err with a null context records the text for m2c_last_error(NULL).
m2c_status set_err(m2c_ctx* c, m2c_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_noctx_error = msg;
  return st;
}

// Parameter check of an EOS (App. B.1 and B.3): stiffened gas (gamma, p_c) with
// gamma > 1; Mie-Grueneisen (rho0, c0, s, Gamma0[, e0[, eta_min]]) with rho0,
// c0, Gamma0 > 0 and s > 1. nullptr when valid, else the reason.
const char* eos_param_error(int type, const double* prm, int nparams) {
  if (type == M2C_EOS_SG) {
    if (nparams < 2 || !(prm[0] > 1.0)) return "SG needs gamma > 1 and p_c";
    return nullptr;
  }
  if (type == M2C_EOS_MG) {
    if (nparams < 4 || nparams > 6) return "MG needs 4 to 6 params";
    if (!(prm[0] > 0.0) || !(prm[1] > 0.0) || !(prm[2] > 1.0) || !(prm[3] > 0.0))
      return "MG needs rho0, c0 > 0, s > 1, Gamma0 > 0";
    return nullptr;
  }
  if (type == M2C_EOS_NASG) {
    if (nparams != 4) return "NASG needs 4 params";
    if (!(prm[0] > 1.0) || !(prm[2] >= 0.0) || !std::isfinite(prm[1]) || !std::isfinite(prm[3]))
      return "NASG needs gamma > 1, b >= 0 and finite p_c, e_c";
    return nullptr;
  }
  if (type == M2C_EOS_JWL) {
    if (nparams != 6) return "JWL needs 6 params";
    if (!(prm[0] > 0.0) || !(prm[3] > 0.0) || !(prm[4] > 0.0) || !(prm[5] > 0.0) || !std::isfinite(prm[1]) ||
        !std::isfinite(prm[2]))
      return "JWL needs omega, R1, R2, rho0 > 0 and finite A1, A2";
    return nullptr;
  }
  return "unknown EOS type";
}

int eos_nparams(int type) {
  return type == M2C_EOS_SG ? 2 : (type == M2C_EOS_NASG ? 4 : 6);
}

// The same for an EOS descriptor of the Riemann entry points (the type's params given).
const char* eos_desc_error(const m2c_eos_desc* e) {
  return eos_param_error(e->type, e->params, eos_nparams(e->type));
}

bool eos_extended(int type) { return type == M2C_EOS_NASG || type == M2C_EOS_JWL; }

// Checks of a grid's sizes, cell edge and boundary conditions shared by
// m2c_init_grid and m2c_residual_noalloc: nullptr when valid, else the reason.
const char* grid_args_error(int nx, int ny, int nz, double h, const int* bc) {
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !bc) return "grid sizes >= 1, h > 0 and bc required";
  if ((long long)nx * ny * nz < 2)  // no axis to move along: no time step
    return "a grid needs an axis with more than one cell";
  if ((long long)nx * ny * nz >= (1ll << 31))  // 32-bit cell indices in some kernels
    return "a grid holds fewer than 2^31 cells";
  const int n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    for (int s = 0; s < 2; ++s) {
      if (bc[2 * a + s] != M2C_BC_TRANSMISSIVE && bc[2 * a + s] != M2C_BC_PERIODIC &&
          bc[2 * a + s] != M2C_BC_SYMMETRY)
        return "unknown boundary condition";
      // the stencils reach two cells across a side: a mirror needs two cells inside
      if (bc[2 * a + s] == M2C_BC_SYMMETRY && n[a] < 2) return "a symmetry side needs 2 cells along its axis";
    }
    if ((bc[2 * a] == M2C_BC_PERIODIC) != (bc[2 * a + 1] == M2C_BC_PERIODIC))
      return "periodic on one side of an axis only";
  }
  return nullptr;
}

// EOS type pair of a grid for the bulk kernel's fixed-type instantiations:
// T0 + 4 T1 when both materials are SG or MG, else -1 (types read at run time).
int material_pair(const Grid& g) {
  const int a = g.eos[0].type, b = g.eos[1].type;
  const bool fixed = (a == M2C_EOS_SG || a == M2C_EOS_MG) && (b == M2C_EOS_SG || b == M2C_EOS_MG);
  return fixed ? a + 4 * b : -1;
}

bool has_symmetry_side(const int* bc) {
  for (int s = 0; s < 6; ++s)
    if (bc[s] == M2C_BC_SYMMETRY) return true;
  return false;
}

// Every entry point that enqueues work on a context, except m2c_step_host itself,
// ends the overlap of m2c_step_host's copies with the previous call's.
inline void end_host_loop(m2c_ctx* c) {
  c->last_W_host = nullptr;
  c->last_phi_host = nullptr;
}

m2c_status cuda_check(m2c_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return M2C_OK;
  return set_err(c, M2C_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// gen: the general instantiation (8-row tiles), for grids with scheme options.
cudaError_t launch_stage(int prec, const Grid* grids, const long long* tiles, int ngrid, long long ntiles, int mode,
                         const LaunchPlan& lp, cudaStream_t s, bool gen = false) {
  if (gen) return launch_stage_gen(prec, grids, tiles, ngrid, ntiles, mode, lp, s);
  if (prec == M2C_FP64) return launch_stage_fp64(grids, tiles, ngrid, ntiles, mode, lp, s);
  return launch_stage_fp32(grids, tiles, ngrid, ntiles, mode, lp, s);
}

void setup_all_stage_kernels() {
  setup_stage_fp64();
  setup_stage_fp32();
  setup_stage_gen();
}

}  // namespace

namespace m2c {

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  return dev < kMaxDevices ? dev : kMaxDevices - 1;
}

int sm_count() {
  static int n[kMaxDevices] = {};
  const int dev = current_device();
  if (!n[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n[dev] = v > 0 ? v : 1;
  }
  return n[dev];
}

}  // namespace m2c

namespace {

void set_tiling(Grid& g, int ty, int tz) {
  g.tiles_x = (g.nx + 31) / 32;
  g.tiles_y = (g.ny + ty - 1) / ty;
  g.tz = std::max(1, std::min(tz, g.nz));
  g.tiles_z = (g.nz + g.tz - 1) / g.tz;
}

long long ntiles_of(const Grid& g) { return (long long)g.tiles_x * g.tiles_y * g.tiles_z; }

m2c_status push_grid(m2c_ctx* c) {
  long long tiles[2] = {0, ntiles_of(c->host)};
  cudaError_t e = cudaMemcpyAsync(c->dev_grid, &c->host, sizeof(Grid), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->dev_tiles, tiles, sizeof(tiles), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  c->dirty = false;
  return cuda_check(c, e, "descriptor upload");
}

// Default tile z-chunk: 64, 32 or 16 planes, the longest that still gives the
// SMs 16 tiles each (the z warm-up of a chunk costs about four planes of
// loads); short grids take one chunk.
// Default tile rows: 16 on the mixed path when 16-row tiles of 16 planes
// still give every SM 8 of them (measured ~3 % faster than 8 rows at 256^3),
// else 8.
int default_rows(const Grid& g) {
  if (g.prec != M2C_MIXED) return 8;
  const long long tiles16 = (long long)((g.nx + 31) / 32) * ((g.ny + 15) / 16) * ((g.nz + 15) / 16);
  return tiles16 >= 8ll * sm_count() ? 16 : 8;
}

int default_tz(const Grid& g, int ty) {
  const long long cols = (long long)((g.nx + 31) / 32) * ((g.ny + ty - 1) / ty);
  const long long want = 16ll * sm_count();
  for (int tz : {64, 32})
    if (g.nz > tz && cols * ((g.nz + tz - 1) / tz) >= want) return tz;
  return g.nz > 16 ? 16 : g.nz;
}

// Event pairs recorded around launches while profiling, tagged with the kernel kind.
enum KernelKind { kKStage = 0, kKFiver, kKFinish, kKReinit, kKPhaseFix, kKEndStep, kKinds };

struct StageEvents {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev;
  std::vector<int>* kind;
  size_t* used;
  bool bulk_only = false;  // time the bulk stage kernel only
  bool skip = false;       // the open pair was not recorded
};

cudaError_t record_pair(StageEvents* pe, bool start, cudaStream_t s, int kind = kKStage) {
  if (!pe) return cudaSuccess;
  if (pe->bulk_only) {
    // only the bulk stage kernel is timed: the end record follows its start record
    if (start && kind != kKStage) {
      pe->skip = true;
      return cudaSuccess;
    }
    if (!start && pe->skip) {
      pe->skip = false;
      return cudaSuccess;
    }
  }
  if (start) {
    if (*pe->used == pe->ev->size()) {
      cudaEvent_t a, b;
      cudaError_t e = cudaEventCreate(&a);
      if (e == cudaSuccess) e = cudaEventCreate(&b);
      if (e != cudaSuccess) return e;
      pe->ev->push_back({a, b});
      pe->kind->push_back(kind);
    }
    (*pe->kind)[*pe->used] = kind;
    return cudaEventRecord((*pe->ev)[*pe->used].first, s);
  }
  cudaError_t e = cudaEventRecord((*pe->ev)[*pe->used].second, s);
  ++*pe->used;
  return e;
}

// reinit: enqueue the reinitialisation kernels (each grid decides on the device
// whether its own step is due); reinit_iters: the largest iteration count.
// rk: the Runge-Kutta scheme of all grids (Sec. 4.3); gen: launch the general
// bulk kernel.
cudaError_t enqueue_step(const Grid* dev_grids, const long long* dev_tiles, int ngrid, long long ntiles, int prec,
                         const LaunchPlan& lp, bool reinit, int reinit_iters, long long nmax, cudaStream_t s,
                         StageEvents* pe = nullptr, int rk = 2, bool gen = false, bool band = false) {
  cudaError_t e;
  const dim3 lg((unsigned)(2 * sm_count()), (unsigned)ngrid);
  const dim3 fg((unsigned)(8 * sm_count()), (unsigned)ngrid);
#define M2C_TIMED(kind, launch)                                     \
  do {                                                              \
    if ((e = record_pair(pe, true, s, kind)) != cudaSuccess) return e; \
    launch;                                                         \
    if ((e = cudaGetLastError()) != cudaSuccess) return e;          \
    if ((e = record_pair(pe, false, s)) != cudaSuccess) return e;   \
  } while (0)
  static const int kModesRk1[1] = {kStage1};
  static const int kModesRk2[2] = {kStage1, kStage2};
  static const int kModesRk3[3] = {kStage1, kStage2of3, kStage3};
  const int* modes = rk == 1 ? kModesRk1 : (rk == 3 ? kModesRk3 : kModesRk2);
  const int nstage = rk == 1 ? 1 : (rk == 3 ? 3 : 2);
  for (int stage = 0; stage < nstage; ++stage) {
    const int mode = modes[stage];
    M2C_TIMED(kKStage, e = launch_stage(prec, dev_grids, dev_tiles, ngrid, ntiles, mode, lp, s, gen); if (e) return e);
    M2C_TIMED(kKFiver, (k_fiver<<<fg, kFiverThreads, 0, s>>>(dev_grids, mode)));
    M2C_TIMED(kKFinish, (k_finish<<<lg, 128, 0, s>>>(dev_grids, mode)));
  }
  if (rk == 1) {
    const dim3 cg((unsigned)std::min<long long>((nmax + 255) / 256, 8ll * sm_count()), (unsigned)ngrid);
    M2C_TIMED(kKFinish, (k_commit_euler<<<cg, 256, 0, s>>>(dev_grids)));
  }
  if (reinit && reinit_iters > 0) {
    const dim3 rg((unsigned)std::min<long long>((nmax + 255) / 256, 8ll * sm_count()), (unsigned)ngrid);
    for (int it = 1; it <= reinit_iters; ++it) {
      if (prec == M2C_FP64) M2C_TIMED(kKReinit, (k_reinit<double><<<rg, 256, 0, s>>>(dev_grids, it)));
      else M2C_TIMED(kKReinit, (k_reinit<float><<<rg, 256, 0, s>>>(dev_grids, it)));
    }
    M2C_TIMED(kKReinit, (k_copy_phi1<<<rg, 256, 0, s>>>(dev_grids)));
  }
  if (band) {
    const dim3 bg((unsigned)std::min<long long>((nmax + 255) / 256, 8ll * sm_count()), (unsigned)ngrid);
    M2C_TIMED(kKReinit, (k_band_clip<<<bg, 256, 0, s>>>(dev_grids)));
  }
  M2C_TIMED(kKPhaseFix, (k_phase_fix<<<lg, 128, 0, s>>>(dev_grids)));
  M2C_TIMED(kKEndStep, (k_end_step<<<(ngrid + 63) / 64, 64, 0, s>>>(dev_grids, ngrid)));
#undef M2C_TIMED
  return cudaGetLastError();
}

}  // namespace

// Wave-speed maximum of the current state for the next step's time step.
static cudaError_t ensure_lam(m2c_ctx* c) {
  cudaError_t e = cudaMemsetAsync(&c->host.ctrl->lam[0], 0, 2 * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return e;
  const dim3 g((unsigned)std::min<long long>((c->host.N + 255) / 256, 8ll * sm_count()), 1);
  k_lam_init<<<g, 256, 0, c->stream>>>(c->dev_grid);
  e = cudaGetLastError();
  if (e == cudaSuccess) c->lam_valid = true;
  return e;
}

namespace {

double lam_to_dt_host(const Grid& g, unsigned long long bits) {
  if (g.dt_fixed > 0.0) return g.dt_fixed;
  double lam;
  std::memcpy(&lam, &bits, sizeof(lam));
  return lam > 0.0 ? g.cfl * g.h / lam : 0.0;
}

}  // namespace

// A batch of grids stepped together: one launch per kernel for all grids.
struct m2c_batch {
  std::vector<m2c_ctx*> ctx;      // largest grid first
  std::vector<Grid> hosts;
  std::vector<long long> tiles;   // prefix sums of the bulk-kernel tiles
  Grid* dev = nullptr;
  long long* dtiles = nullptr;
  unsigned long long* counter = nullptr;
  LaunchPlan lp;
  int prec = 0;
  cudaStream_t stream = nullptr;
  long long step = 0, nmax = 1;
  int reinit_every = 10, reinit_iters = 5, graph_steps = 0;
  int rk = 2;        // Runge-Kutta scheme of every grid
  bool gen = false;  // some grid has scheme options: the general bulk kernel
  bool band = false; // some grid has a narrow-band level set
};

extern "C" {

const char* m2c_status_string(int s) {
  switch (s) {
    case M2C_OK: return "ok";
    case M2C_EINVAL: return "invalid argument";
    case M2C_ENOMEM: return "workspace too small";
    case M2C_ECUDA: return "CUDA error";
    case M2C_ENOCONV: return "Riemann solver did not converge";
    case M2C_ENONPHYS: return "non-physical state";
    case M2C_EVACUUM: return "vacuum in the Riemann problem";
    case M2C_ETIMEOUT: return "device wait timed out";
    case M2C_EOVERFLOW: return "interface work list overflow";
    default: return "unknown status";
  }
}

size_t m2c_workspace_bytes(int nx, int ny, int nz, int precision) {
  (void)precision;
  if (nx < 1 || ny < 1 || nz < 1) return 0;
  return layout_for((long long)nx * ny * nz).total;
}

size_t m2c_workspace_bytes_rk(int nx, int ny, int nz, int precision, int rk) {
  (void)precision;
  if (nx < 1 || ny < 1 || nz < 1 || rk < 1 || rk > 3) return 0;
  return layout_for((long long)nx * ny * nz, rk).total;
}

m2c_status m2c_init_grid(m2c_ctx** out, int nx, int ny, int nz, const double lo[3], double h, const int bc[6],
                         int precision, void* workspace, size_t ws_bytes, void* stream) {
  (void)lo;
  g_noctx_error.clear();
  if (!out) return set_err(nullptr, M2C_EINVAL, "out is NULL");
  *out = nullptr;
  if (const char* why = grid_args_error(nx, ny, nz, h, bc)) return set_err(nullptr, M2C_EINVAL, why);
  if (!workspace) return set_err(nullptr, M2C_EINVAL, "workspace required");
  if (precision != M2C_FP64 && precision != M2C_MIXED) return set_err(nullptr, M2C_EINVAL, "unknown precision");
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign)
    return set_err(nullptr, M2C_EINVAL, "workspace is not 256-byte aligned");
  const long long N = (long long)nx * ny * nz;
  const Layout L = layout_for(N);
  if (ws_bytes < L.total) return set_err(nullptr, M2C_ENOMEM, "workspace smaller than m2c_workspace_bytes()");
  m2c_ctx* c = new (std::nothrow) m2c_ctx();
  if (!c) return set_err(nullptr, M2C_ENOMEM, "out of host memory for the context");
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  Grid& g = c->host;
  std::memset(&g, 0, sizeof(g));
  g.nx = nx; g.ny = ny; g.nz = nz; g.N = N;
  for (int s = 0; s < 6; ++s) g.bc[s] = bc[s];
  g.active[0] = nx > 1; g.active[1] = ny > 1; g.active[2] = nz > 1;
  g.prec = precision;
  g.h = h; g.inv_h = 1.0 / h; g.cfl = 0.5;
  g.W1 = reinterpret_cast<double*>(ws + L.W1);
  g.phi1 = reinterpret_cast<double*>(ws + L.phi1);
  g.phiC = reinterpret_cast<double*>(ws + L.phiC);
  g.id = ws + L.id;
  g.cell_slot = reinterpret_cast<int*>(ws + L.slot);
  g.faces = reinterpret_cast<IfFace*>(ws + L.faces);
  g.cells = reinterpret_cast<IfCell*>(ws + L.cells);
  g.flips = reinterpret_cast<long long*>(ws + L.flips);
  g.face_cap = L.face_cap; g.cell_cap = L.cell_cap; g.flip_cap = L.flip_cap;
  g.ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
  g.pstar = reinterpret_cast<double*>(ws + L.pstar);
  g.rk = 2;
  g.limiter = M2C_LIM_VAN_ALBADA;
  g.flux = M2C_FLUX_HLLC;
  g.mc_alpha = 1.2;
  g.dt_fixed = 0.0;
  g.geom = M2C_GEOM_CARTESIAN;
  g.x0 = 0.0;
  g.general = has_symmetry_side(bc) ? 1 : 0;  // mirror loads: the general kernel
  const Layout L3 = layout_for(N, 3);
  if (ws_bytes >= L3.total) {  // room for the second stage state of TVD RK3
    g.W2 = reinterpret_cast<double*>(ws + L3.W2);
    g.phi2 = reinterpret_cast<double*>(ws + L3.phi2);
  }
  c->ws_bytes = ws_bytes;
  c->dev_grid = reinterpret_cast<Grid*>(ws + L.grid);
  c->dev_tiles = reinterpret_cast<long long*>(ws + L.tiles);
  c->stream = static_cast<cudaStream_t>(stream);
  setup_all_stage_kernels();
  c->ty = g.general ? 8 : default_rows(g);
  set_tiling(g, c->ty, default_tz(g, c->ty));
  c->reinit_every = 10;
  c->reinit_iters = 5;
  g.reinit_every = 10;
  g.reinit_iters = 5;
  c->host_step = 0;
  c->has_state = false;
  c->eos_set[0] = c->eos_set[1] = false;
  c->lam_valid = false;
  c->profiling = false;
  c->profile_bulk_only = false;
  c->ev_used = 0;
  // a failure here leaves no context: its text goes to m2c_last_error(NULL)
  cudaError_t e = cudaMemsetAsync(g.ctrl, 0, sizeof(Ctrl), c->stream);
  if (e != cudaSuccess) {
    delete c;
    return set_err(nullptr, M2C_ECUDA, std::string("control block reset: ") + cudaGetErrorString(e));
  }
  m2c_status st = push_grid(c);
  if (st != M2C_OK) {
    const std::string why = c->err;
    delete c;
    return set_err(nullptr, st, why);
  }
  *out = c;
  return M2C_OK;
}

static void update_general(m2c_ctx* c);

m2c_status m2c_set_eos(m2c_ctx* c, int material, int type, const double* params, int nparams) {
  if (!c) return M2C_EINVAL;
  if (material < 0 || material > 1 || !params) return set_err(c, M2C_EINVAL, "bad material or params");
  if (const char* why = eos_param_error(type, params, nparams)) return set_err(c, M2C_EINVAL, why);
  double prm[6] = {0, 0, 0, 0, 0, type == M2C_EOS_MG ? -INFINITY : 0.0};
  for (int i = 0; i < (type == M2C_EOS_SG ? 2 : nparams); ++i) prm[i] = params[i];
  c->host.eos[material] = make_eos<double>(type, prm);
  c->host.eosf[material] = make_eos<float>(type, prm);
  c->eos_set[material] = true;
  update_general(c);
  return push_grid(c);
}

m2c_status m2c_set_scheme(m2c_ctx* c, double cfl, int reinit_every, int reinit_iters) {
  if (!c) return M2C_EINVAL;
  if (!(cfl > 0.0) || reinit_every < 0 || reinit_iters < 0) return set_err(c, M2C_EINVAL, "bad scheme parameters");
  c->host.cfl = cfl;
  c->reinit_every = reinit_every;
  c->reinit_iters = reinit_iters;
  c->host.reinit_every = reinit_every;
  c->host.reinit_iters = reinit_iters;
  return push_grid(c);
}

// The general bulk kernel serves every grid with a scheme option, a symmetry
// side or a NASG / JWL material; it runs 8-row tiles.
static void update_general(m2c_ctx* c) {
  Grid& g = c->host;
  g.general = (g.rk == 3 || g.limiter != M2C_LIM_VAN_ALBADA || g.flux != M2C_FLUX_HLLC ||
               g.geom != M2C_GEOM_CARTESIAN || has_symmetry_side(g.bc) || eos_extended(g.eos[0].type) ||
               eos_extended(g.eos[1].type) || g.band_gamma > 0.0) ? 1 : 0;
  if (g.general && c->ty != 8) {
    c->ty = 8;
    set_tiling(g, 8, default_tz(g, 8));
  }
}

m2c_status m2c_set_options(m2c_ctx* c, const m2c_options* o) {
  if (!c) return M2C_EINVAL;
  if (!o) return set_err(c, M2C_EINVAL, "options are NULL");
  if (o->rk < 1 || o->rk > 3) return set_err(c, M2C_EINVAL, "rk must be 1, 2 or 3");
  if (o->limiter != M2C_LIM_VAN_ALBADA && o->limiter != M2C_LIM_MC) return set_err(c, M2C_EINVAL, "unknown limiter");
  if (o->flux != M2C_FLUX_HLLC && o->flux != M2C_FLUX_LLF) return set_err(c, M2C_EINVAL, "unknown flux");
  if (o->limiter == M2C_LIM_MC && !(o->mc_alpha >= 1.0 && o->mc_alpha <= 2.0))
    return set_err(c, M2C_EINVAL, "the MC limiter needs 1 <= alpha <= 2");
  if (!(o->dt_fixed >= 0.0) || !std::isfinite(o->dt_fixed)) return set_err(c, M2C_EINVAL, "dt_fixed must be >= 0");
  if (o->geom != M2C_GEOM_CARTESIAN && o->geom != M2C_GEOM_CYLINDRICAL && o->geom != M2C_GEOM_SPHERICAL)
    return set_err(c, M2C_EINVAL, "unknown geometry");
  if (o->geom != M2C_GEOM_CARTESIAN && !(o->x0 >= 0.0 && std::isfinite(o->x0)))
    return set_err(c, M2C_EINVAL, "the radius x0 of the first face must be >= 0");
  if (o->geom == M2C_GEOM_SPHERICAL && (c->host.ny != 1 || c->host.nz != 1))
    return set_err(c, M2C_EINVAL, "the spherical form is one-dimensional (ny = nz = 1)");
  if (o->geom == M2C_GEOM_CYLINDRICAL && c->host.ny != 1)
    return set_err(c, M2C_EINVAL, "the cylindrical form is (r, z): ny = 1");
  if (!(o->band_gamma >= 0.0) || (o->band_gamma > 0.0 && !(o->band_beta > 0.0 && o->band_beta < o->band_gamma)))
    return set_err(c, M2C_EINVAL, "a narrow band needs 0 < band_beta < band_gamma (cells)");
  if (o->rk == 3 && !c->host.W2)
    return set_err(c, M2C_ENOMEM, "TVD RK3 needs a workspace of m2c_workspace_bytes_rk(nx, ny, nz, precision, 3)");
  Grid& g = c->host;
  g.rk = o->rk;
  g.limiter = o->limiter;
  g.flux = o->flux;
  g.mc_alpha = o->limiter == M2C_LIM_MC ? o->mc_alpha : 1.2;
  g.dt_fixed = o->dt_fixed;
  g.geom = o->geom;
  g.x0 = o->geom != M2C_GEOM_CARTESIAN ? o->x0 : 0.0;
  g.band_beta = o->band_gamma > 0.0 ? o->band_beta * g.h : 0.0;
  g.band_gamma = o->band_gamma > 0.0 ? o->band_gamma * g.h : 0.0;
  update_general(c);
  return push_grid(c);
}

m2c_status m2c_set_riemann_start(m2c_ctx* c, int fp32_start) {
  if (!c || (fp32_start != 0 && fp32_start != 1)) return M2C_EINVAL;
  if (fp32_start && c->host.prec != M2C_MIXED)
    return set_err(c, M2C_EINVAL, "the FP32 Riemann start is an option of M2C_MIXED grids");
  c->host.riemann_fp32_start = fp32_start;
  return push_grid(c);
}

m2c_status m2c_set_tiling(m2c_ctx* c, int tile_rows, int tile_z) {
  if (!c || (tile_rows != 4 && tile_rows != 8 && tile_rows != 16) || tile_z < 0) return M2C_EINVAL;
  if (tile_rows == 16 && c->host.prec == M2C_FP64) return set_err(c, M2C_EINVAL, "FP64 tiles have 4 or 8 rows");
  if (c->host.general && tile_rows != 8)
    return set_err(c, M2C_EINVAL, "grids with scheme options run 8-row tiles");
  c->ty = tile_rows;
  set_tiling(c->host, c->ty, tile_z > 0 ? tile_z : default_tz(c->host, c->ty));
  return push_grid(c);
}

m2c_status m2c_set_state(m2c_ctx* c, double* W, double* phi, double t, long step) {
  if (!c) return M2C_EINVAL;
  end_host_loop(c);
  if (!W || !phi) return set_err(c, M2C_EINVAL, "null state");
  if (!c->eos_set[0] || !c->eos_set[1]) return set_err(c, M2C_EINVAL, "set both EOS first");
  c->host.W = W;
  c->host.phi = phi;
  m2c_status st = push_grid(c);
  if (st) return st;
  Ctrl init;
  std::memset(&init, 0, sizeof(init));
  init.t = t;
  init.step = step;
  init.err_cell = -1;
  cudaError_t e = cudaMemcpyAsync(c->host.ctrl, &init, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "set_state");
  // a new state starts the FIVER warm-start cache empty (all bits set: NaN)
  e = cudaMemsetAsync(c->host.pstar, 0xff, sizeof(double) * 3 * (size_t)c->host.N, c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "set_state");
  c->host_step = step;
  c->has_state = true;
  c->lam_valid = false;  // the first time step is reduced at the next m2c_step
  e = cudaStreamSynchronize(c->stream);
  return cuda_check(c, e, "set_state");
}

m2c_status m2c_prims_to_state(m2c_ctx* c, const double* prims) {
  if (!c || !prims) return M2C_EINVAL;
  end_host_loop(c);
  if (!c->has_state) return set_err(c, M2C_EINVAL, "set_state first (W and phi buffers)");
  const dim3 g((unsigned)std::min<long long>((c->host.N + 255) / 256, 8ll * sm_count()), 1);
  k_prims_to_state<<<g, 256, 0, c->stream>>>(c->dev_grid, prims);
  c->lam_valid = false;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_check(c, e, "prims_to_state");
}

m2c_status m2c_state_to_prims(m2c_ctx* c, double* prims) {
  if (!c || !prims) return M2C_EINVAL;
  end_host_loop(c);
  if (!c->has_state) return set_err(c, M2C_EINVAL, "set_state first");
  const dim3 g((unsigned)std::min<long long>((c->host.N + 255) / 256, 8ll * sm_count()), 1);
  k_state_to_prims<<<g, 256, 0, c->stream>>>(c->dev_grid, prims);
  return cuda_check(c, cudaGetLastError(), "state_to_prims");
}

m2c_status m2c_upload_state(m2c_ctx* c, const double* W_host, const double* phi_host) {
  if (!c || !W_host || !phi_host) return M2C_EINVAL;
  end_host_loop(c);
  if (!c->has_state) return set_err(c, M2C_EINVAL, "set_state first");
  const size_t N = (size_t)c->host.N;
  cudaError_t e = cudaMemcpyAsync(c->host.W, W_host, 5 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->host.phi, phi_host, N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  c->lam_valid = false;
  return cuda_check(c, e, "upload_state");
}

m2c_status m2c_download_state(m2c_ctx* c, double* W_host, double* phi_host) {
  if (!c || !W_host || !phi_host) return M2C_EINVAL;
  end_host_loop(c);
  if (!c->has_state) return set_err(c, M2C_EINVAL, "set_state first");
  const size_t N = (size_t)c->host.N;
  cudaError_t e = cudaMemcpyAsync(W_host, c->host.W, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(phi_host, c->host.phi, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_check(c, e, "download_state");
}

m2c_status m2c_step_host(m2c_ctx* c, double* W_host, double* phi_host, int nsteps) {
  if (!c || !W_host || !phi_host || nsteps < 0) return M2C_EINVAL;
  if (!c->has_state) return set_err(c, M2C_EINVAL, "set_state first");
  cudaError_t e = cudaSuccess;
  if (!c->copy_in) {
    e = cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&c->down_ev[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->up_ev[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_check(c, e, "step_host set-up");
  }
  const size_t N = (size_t)c->host.N;
  const bool same = W_host == c->last_W_host && phi_host == c->last_phi_host;
  auto host_of = [&](int k) { return k < 5 ? W_host + (size_t)k * N : phi_host; };
  auto dev_of = [&](int k) { return k < 5 ? c->host.W + (size_t)k * N : c->host.phi; };
  // the uploads may not overwrite the state while work enqueued before this call
  // still uses it: after a call on the same host arrays with nothing enqueued on
  // the context since (every other entry point that enqueues work clears
  // last_W_host), component k waits only for that call's download of it;
  // otherwise the copy stream waits for everything enqueued on the context's stream
  if (!same) {
    e = cudaEventRecord(c->up_ev[0], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_in, c->up_ev[0], 0);
  }
  for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
    if (same) e = cudaStreamWaitEvent(c->copy_in, c->down_ev[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dev_of(k), host_of(k), N * sizeof(double), cudaMemcpyHostToDevice, c->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(c->up_ev[k], c->copy_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->up_ev[k], 0);
  }
  if (e != cudaSuccess) return cuda_check(c, e, "step_host upload");
  c->lam_valid = false;
  m2c_status st = m2c_step(c, nsteps);
  if (st) return st;
  for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
    e = cudaMemcpyAsync(host_of(k), dev_of(k), N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->down_ev[k], c->stream);
  }
  c->last_W_host = W_host;
  c->last_phi_host = phi_host;
  return cuda_check(c, e, "step_host download");
}

m2c_status m2c_step(m2c_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return M2C_EINVAL;
  end_host_loop(c);
  if (!c->has_state) return set_err(c, M2C_EINVAL, "no state");
  if (!c->lam_valid && nsteps > 0) {
    cudaError_t e = ensure_lam(c);
    if (e != cudaSuccess) return cuda_check(c, e, "first time step");
  }
  for (int n = 0; n < nsteps; ++n) {
    const bool re = c->reinit_every > 0 && (c->host_step + 1) % c->reinit_every == 0;
    StageEvents pe{&c->ev, &c->ev_kind, &c->ev_used, c->profile_bulk_only, false};
    LaunchPlan lp;
    lp.ty = c->ty;
    lp.mats = material_pair(c->host);
    cudaError_t e = enqueue_step(c->dev_grid, c->dev_tiles, 1, ntiles_of(c->host), c->host.prec, lp, re,
                                 c->reinit_iters, c->host.N, c->stream, c->profiling ? &pe : nullptr, c->host.rk,
                                 c->host.general != 0, c->host.band_gamma > 0.0);
    if (e != cudaSuccess) return cuda_check(c, e, "step launch");
    ++c->host_step;
  }
  return M2C_OK;
}

size_t m2c_batch_workspace_bytes(int k) {
  if (k < 1) return 0;
  return align_up(sizeof(Grid) * (size_t)k) + align_up(sizeof(long long) * (size_t)(k + 1)) + kAlign;
}

m2c_status m2c_batch_create(m2c_batch** out, m2c_ctx** v, int k, void* workspace, size_t bytes, const int tuning[4]) {
  if (!out || !v || k < 1 || !workspace) return M2C_EINVAL;
  *out = nullptr;
  if (bytes < m2c_batch_workspace_bytes(k) || reinterpret_cast<uintptr_t>(workspace) % kAlign) return M2C_EINVAL;
  for (int i = 0; i < k; ++i) {
    if (!v[i] || !v[i]->has_state) return M2C_EINVAL;
    if (v[i]->host.prec != v[0]->host.prec) return set_err(v[0], M2C_EINVAL, "one precision per batch");
    if (v[i]->host.rk != v[0]->host.rk) return set_err(v[0], M2C_EINVAL, "one Runge-Kutta scheme per batch");
  }
  bool gen = false;
  for (int i = 0; i < k; ++i) gen = gen || v[i]->host.general != 0;
  int ty = 8, tz = 0, sched = 0, bpsm = 0;
  if (tuning) {
    ty = tuning[0] == 4 ? 4 : (tuning[0] == 16 && v[0]->host.prec == M2C_MIXED ? 16 : 8);
    tz = std::max(0, tuning[1]);
    sched = tuning[2] == 1 ? 1 : 0;
    bpsm = std::max(0, tuning[3]);
  }
  if (gen) ty = 8;  // the general kernel runs 8-row tiles
  m2c_batch* b = new (std::nothrow) m2c_batch();
  if (!b) return M2C_ENOMEM;
  // largest grids first, so that the longest tiles start early
  std::vector<int> order(k);
  for (int i = 0; i < k; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return v[a]->host.N > v[c]->host.N; });
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  b->dev = reinterpret_cast<Grid*>(ws);
  b->dtiles = reinterpret_cast<long long*>(ws + align_up(sizeof(Grid) * (size_t)k));
  b->counter = reinterpret_cast<unsigned long long*>(ws + align_up(sizeof(Grid) * (size_t)k) +
                                                     align_up(sizeof(long long) * (size_t)(k + 1)));
  b->tiles.assign(k + 1, 0);
  b->nmax = 1;
  for (int i = 0; i < k; ++i) {
    m2c_ctx* c = v[order[i]];
    b->ctx.push_back(c);
    Grid g = c->host;
    set_tiling(g, ty, tz > 0 ? tz : default_tz(g, ty));
    b->hosts.push_back(g);
    b->tiles[i + 1] = b->tiles[i] + ntiles_of(g);
    b->nmax = std::max(b->nmax, g.N);
  }
  b->lp.ty = ty;
  b->lp.sched = sched;
  b->lp.blocks_per_sm = bpsm;
  b->lp.counter = b->counter;
  b->lp.mats = material_pair(b->hosts[0]);
  for (int i = 1; i < k; ++i)
    if (material_pair(b->hosts[i]) != b->lp.mats) b->lp.mats = -1;
  b->prec = v[0]->host.prec;
  b->rk = v[0]->host.rk;
  b->gen = gen;
  for (int i = 0; i < k; ++i) b->band = b->band || v[i]->host.band_gamma > 0.0;
  b->stream = v[0]->stream;
  b->step = v[0]->host_step;
  b->reinit_every = v[0]->reinit_every;
  b->reinit_iters = 0;
  for (int i = 0; i < k; ++i)
    if (v[i]->reinit_every > 0) b->reinit_iters = std::max(b->reinit_iters, v[i]->reinit_iters);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < k && e == cudaSuccess; ++i) {
    m2c_ctx* c = b->ctx[i];
    if (!c->lam_valid) {
      e = ensure_lam(c);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->dev, b->hosts.data(), sizeof(Grid) * k, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->dtiles, b->tiles.data(), sizeof(long long) * (k + 1), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    delete b;
    return cuda_check(v[0], e, "batch_create");
  }
  *out = b;
  return M2C_OK;
}

static m2c_status batch_enqueue(m2c_batch* b, int nsteps, cudaStream_t s) {
  const int k = (int)b->ctx.size();
  for (int n = 0; n < nsteps; ++n) {
    // grids of a batch may be at different steps: the reinitialisation kernels
    // are enqueued every step and each grid checks its own schedule
    cudaError_t e = enqueue_step(b->dev, b->dtiles, k, b->tiles[k], b->prec, b->lp, b->reinit_iters > 0,
                                 b->reinit_iters, b->nmax, s, nullptr, b->rk, b->gen, b->band);
    if (e != cudaSuccess) return cuda_check(b->ctx[0], e, "batch step launch");
    ++b->step;
    for (m2c_ctx* c : b->ctx) ++c->host_step;
  }
  return M2C_OK;
}

m2c_status m2c_batch_step(m2c_batch* b, int nsteps) {
  if (!b || nsteps < 0) return M2C_EINVAL;
  for (m2c_ctx* c : b->ctx) end_host_loop(c);
  return batch_enqueue(b, nsteps, b->stream);
}

m2c_status m2c_batch_capture(m2c_batch* b, int nsteps, void** graph_exec) {
  if (!b || nsteps < 1 || !graph_exec) return M2C_EINVAL;
  *graph_exec = nullptr;
  cudaStream_t s;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_check(b->ctx[0], e, "capture stream");
  const long long step0 = b->step;
  std::vector<long long> hs0;
  for (m2c_ctx* c : b->ctx) hs0.push_back(c->host_step);
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  m2c_status st = M2C_OK;
  if (e == cudaSuccess) st = batch_enqueue(b, nsteps, s);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  // the captured steps run when the graph is launched: the schedule counters advance then
  b->step = step0;
  for (size_t i = 0; i < b->ctx.size(); ++i) b->ctx[i]->host_step = hs0[i];
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && st == M2C_OK && e2 == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(s);
  if (st != M2C_OK) return st;
  if (e != cudaSuccess || e2 != cudaSuccess) return cuda_check(b->ctx[0], e != cudaSuccess ? e : e2, "graph capture");
  b->graph_steps = nsteps;
  *graph_exec = exec;
  return M2C_OK;
}

m2c_status m2c_batch_launch_graph(m2c_batch* b, void* graph_exec) {
  if (!b || !graph_exec) return M2C_EINVAL;
  for (m2c_ctx* c : b->ctx) end_host_loop(c);
  cudaError_t e = cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), b->stream);
  if (e != cudaSuccess) return cuda_check(b->ctx[0], e, "graph launch");
  b->step += b->graph_steps;
  for (m2c_ctx* c : b->ctx) c->host_step += b->graph_steps;
  return M2C_OK;
}

void m2c_graph_destroy(void* graph_exec) {
  if (graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
}

void m2c_batch_destroy(m2c_batch* b) { delete b; }

m2c_status m2c_residual(m2c_ctx* c, double* R, double* L) {
  if (!c || !R || !L) return M2C_EINVAL;
  end_host_loop(c);
  if (!c->has_state) return set_err(c, M2C_EINVAL, "no state");
  c->host.resR = R;
  c->host.resL = L;
  m2c_status st = push_grid(c);
  if (st) return st;
  LaunchPlan lp;
  lp.ty = c->ty;
  lp.mats = material_pair(c->host);
  cudaError_t e = launch_stage(c->host.prec, c->dev_grid, c->dev_tiles, 1, ntiles_of(c->host), kResidual, lp,
                               c->stream, c->host.general != 0);
  if (e == cudaSuccess) {
    const dim3 lg((unsigned)(2 * sm_count()), 1);
    k_fiver<<<dim3((unsigned)(8 * sm_count()), 1), kFiverThreads, 0, c->stream>>>(c->dev_grid, kResidual);
    k_finish<<<lg, 128, 0, c->stream>>>(c->dev_grid, kResidual);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(&c->host.ctrl->nface[0], 0, 3 * sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&c->host.ctrl->ncell[0], 0, 3 * sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_check(c, e, "residual");
}

m2c_status m2c_sync(m2c_ctx* c, double* t, long* steps, long* err_cell) {
  if (!c) return M2C_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "sync");
  Ctrl h;
  e = cudaMemcpy(&h, c->host.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_check(c, e, "sync");
  if (t) *t = h.t;
  if (steps) *steps = (long)h.step;
  if (err_cell) *err_cell = h.err ? (long)h.err_cell : -1;
  if (h.err) {
    const int zero[1] = {0};
    cudaMemcpy(&c->host.ctrl->err, zero, sizeof(int), cudaMemcpyHostToDevice);
    return set_err(c, (m2c_status)h.err, std::string("device: ") + m2c_status_string(h.err) + " at cell " +
                                             std::to_string(h.err_cell));
  }
  return M2C_OK;
}

m2c_status m2c_get_stats(m2c_ctx* c, m2c_stats* out) {
  if (!c || !out) return M2C_EINVAL;
  Ctrl h;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(&h, c->host.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_check(c, e, "get_stats");
  out->interface_faces = (long)h.stat_faces;
  out->interface_cells = (long)h.stat_cells;
  out->flipped_cells = (long)h.stat_flips;
  out->dt = h.step == 0 ? lam_to_dt_host(c->host, h.lam[0]) : h.stat_dt;
  return M2C_OK;
}

// Staging layout of the host-array Riemann entry points in the caller's
// workspace: L (3n), R (3n), out (4n) doubles, iters (n) and status (n) ints.
static size_t riemann_ws_layout(long long n, size_t off[5]) {
  size_t o = 0;
  off[0] = o; o = align_up(o + sizeof(double) * 3 * (size_t)n);
  off[1] = o; o = align_up(o + sizeof(double) * 3 * (size_t)n);
  off[2] = o; o = align_up(o + sizeof(double) * 4 * (size_t)n);
  off[3] = o; o = align_up(o + sizeof(int) * (size_t)n);
  off[4] = o; o = align_up(o + sizeof(int) * (size_t)n);
  return o;
}

size_t m2c_riemann_workspace_bytes(int n) {
  if (n < 1) n = 1;
  size_t off[5];
  return riemann_ws_layout(n, off);
}

static m2c_status solve_riemann_batch(int mixed, int n, const m2c_eos_desc* eosL, const double* L,
                                      const m2c_eos_desc* eosR, const double* R, double* out, int* iters, int* status,
                                      int on_device, void* workspace, size_t ws_bytes, void* stream) {
  g_noctx_error.clear();
  if (n < 0 || !eosL || !eosR || !L || !R || !out) return set_err(nullptr, M2C_EINVAL, "bad batch arguments");
  if (const char* why = eos_desc_error(eosL)) return set_err(nullptr, M2C_EINVAL, std::string("left EOS: ") + why);
  if (const char* why = eos_desc_error(eosR)) return set_err(nullptr, M2C_EINVAL, std::string("right EOS: ") + why);
  if (n == 0) return M2C_OK;
  size_t off[5];
  if (!on_device) {
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlign)
      return set_err(nullptr, M2C_EINVAL, "host arrays need a 256-byte aligned device workspace");
    if (ws_bytes < riemann_ws_layout(n, off))
      return set_err(nullptr, M2C_ENOMEM, "workspace smaller than m2c_riemann_workspace_bytes(n)");
  }
  double pl[6] = {0, 0, 0, 0, 0, -INFINITY}, pr[6] = {0, 0, 0, 0, 0, -INFINITY};
  for (int i = 0; i < 6; ++i) {
    pl[i] = eosL->params[i];
    pr[i] = eosR->params[i];
  }
  const EosDev qL = make_eos_dev(eosL->type, pl), qR = make_eos_dev(eosR->type, pr);
  const EosP<float> qLf = make_eos<float>(eosL->type, pl), qRf = make_eos<float>(eosR->type, pr);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int threads = 128;
  const int blocks = (int)std::min<long long>((n + threads - 1) / threads, 4ll * sm_count());
  if (on_device) {
    k_riemann_batch<<<blocks, threads, 0, s>>>(n, qL, L, qR, R, out, iters, status, mixed, qLf, qRf);
    return cudaGetLastError() == cudaSuccess ? M2C_OK : set_err(nullptr, M2C_ECUDA, "Riemann batch launch");
  }
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* dL = reinterpret_cast<double*>(ws + off[0]);
  double* dR = reinterpret_cast<double*>(ws + off[1]);
  double* dO = reinterpret_cast<double*>(ws + off[2]);
  int* dI = reinterpret_cast<int*>(ws + off[3]);
  int* dS = reinterpret_cast<int*>(ws + off[4]);
  std::vector<int> hs(n);
  cudaError_t e = cudaMemcpyAsync(dL, L, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dR, R, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_riemann_batch<<<blocks, threads, 0, s>>>(n, qL, dL, qR, dR, dO, dI, dS, mixed, qLf, qRf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dO, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), dS, sizeof(int) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && iters) e = cudaMemcpyAsync(iters, dI, sizeof(int) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_err(nullptr, M2C_ECUDA, std::string("Riemann batch: ") + cudaGetErrorString(e));
  if (status) std::memcpy(status, hs.data(), sizeof(int) * n);
  for (int i = 0; i < n; ++i)
    if (hs[i]) return set_err(nullptr, (m2c_status)hs[i], "problem " + std::to_string(i) + ": " + m2c_status_string(hs[i]));
  return M2C_OK;
}

m2c_status m2c_solve_riemann(int n, const m2c_eos_desc* eosL, const double* L, const m2c_eos_desc* eosR,
                             const double* R, double* out, int* iters, int* status, int on_device, void* workspace,
                             size_t ws_bytes, void* stream) {
  return solve_riemann_batch(0, n, eosL, L, eosR, R, out, iters, status, on_device, workspace, ws_bytes, stream);
}

m2c_status m2c_solve_riemann_mixed(int n, const m2c_eos_desc* eosL, const double* L, const m2c_eos_desc* eosR,
                                   const double* R, double* out, int* iters, int* status, int on_device,
                                   void* workspace, size_t ws_bytes, void* stream) {
  return solve_riemann_batch(1, n, eosL, L, eosR, R, out, iters, status, on_device, workspace, ws_bytes, stream);
}

m2c_status m2c_shock_state(const m2c_eos_desc* eos, const double w[3], double p1, double out[3], void* workspace,
                           size_t ws_bytes, void* stream) {
  g_noctx_error.clear();
  if (!eos || !w || !out) return set_err(nullptr, M2C_EINVAL, "bad shock-state arguments");
  if (const char* why = eos_desc_error(eos)) return set_err(nullptr, M2C_EINVAL, why);
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % kAlign)
    return set_err(nullptr, M2C_EINVAL, "a 256-byte aligned device workspace is required");
  if (ws_bytes < m2c_riemann_workspace_bytes(1))
    return set_err(nullptr, M2C_ENOMEM, "workspace smaller than m2c_riemann_workspace_bytes(1)");
  double prm[6];
  for (int i = 0; i < 6; ++i) prm[i] = eos->params[i];
  const EosDev q = make_eos_dev(eos->type, prm);
  double* d = static_cast<double*>(workspace);
  int* ds = reinterpret_cast<int*>(d + 3);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_shock_state<<<1, 1, 0, s>>>(q, w[0], w[1], w[2], p1, d, ds);
  double h[4];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_err(nullptr, M2C_ECUDA, std::string("shock state: ") + cudaGetErrorString(e));
  int st;
  std::memcpy(&st, &h[3], sizeof(int));
  if (st) return set_err(nullptr, (m2c_status)st, m2c_status_string(st));
  out[0] = h[0]; out[1] = h[1]; out[2] = h[2];
  return M2C_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free stage residual.
//
// For callers that cannot allocate device memory (a host application whose
// device memory is handed out by its own pool and must not grow, code that
// may not trigger the implicit device synchronisation of cudaMalloc/cudaFree,
// or code that runs where the CUDA allocator is off limits), this entry point
// computes the same stage residual as m2c_residual with no context and no
// workspace: its scratch (grid descriptor, control block, material ids, the
// interface work lists) is one file-scope device array of fixed size, which
// every GPU that loads this library holds until the process exits. Host code
// must not pass the array's name to a kernel (in host code it is only a
// stand-in); its device address is looked up once per device, with that
// device current, by the first call on the device.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace m2c {
constexpr long long kNoAllocMaxCells = M2C_NOALLOC_MAX_CELLS;
constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr long long kNoAllocFaceCap = kNoAllocMaxCells / 4 > 4096 ? kNoAllocMaxCells / 4 : 4096;
constexpr long long kNoAllocCellCap = kNoAllocMaxCells / 8 > 2048 ? kNoAllocMaxCells / 8 : 2048;
constexpr size_t kNaGrid = 0;
constexpr size_t kNaTiles = na_align(kNaGrid + sizeof(Grid));
constexpr size_t kNaCtrl = na_align(kNaTiles + 2 * sizeof(long long));
constexpr size_t kNaId = na_align(kNaCtrl + sizeof(Ctrl));
constexpr size_t kNaSlot = na_align(kNaId + (size_t)kNoAllocMaxCells);
constexpr size_t kNaFaces = na_align(kNaSlot + sizeof(int) * (size_t)kNoAllocMaxCells);
constexpr size_t kNaCells = na_align(kNaFaces + sizeof(IfFace) * (size_t)kNoAllocFaceCap);
constexpr size_t kNaBytes = na_align(kNaCells + sizeof(IfCell) * (size_t)kNoAllocCellCap);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];
}  // namespace m2c

namespace {
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};
m2c_status noalloc_fail(m2c_status st, const std::string& msg) {
  g_noctx_error = msg;
  return st;
}

// Device address of the scratch array on the current device, looked up once.
m2c_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(M2C_ECUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, m2c::g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(M2C_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return M2C_OK;
}
}  // namespace

extern "C" {

size_t m2c_residual_noalloc_scratch_bytes(void) { return m2c::kNaBytes; }

m2c_status m2c_residual_noalloc(int nx, int ny, int nz, double h, const int bc[6], const m2c_eos_desc* eos0,
                                const m2c_eos_desc* eos1, int precision, const double* W, const double* phi,
                                double* R, double* L, void* stream) {
  g_noctx_error.clear();  // keeps its capacity: no allocation
  if (!eos0 || !eos1 || !W || !phi || !R || !L) return noalloc_fail(M2C_EINVAL, "m2c_residual_noalloc: bad argument");
  if (const char* why = grid_args_error(nx, ny, nz, h, bc))
    return noalloc_fail(M2C_EINVAL, std::string("m2c_residual_noalloc: ") + why);
  if (precision != M2C_FP64 && precision != M2C_MIXED)
    return noalloc_fail(M2C_EINVAL, "m2c_residual_noalloc: bad precision");
  if (has_symmetry_side(bc))
    return noalloc_fail(M2C_EINVAL, "m2c_residual_noalloc: transmissive and periodic sides only");
  if (eos_extended(eos0->type) || eos_extended(eos1->type))
    return noalloc_fail(M2C_EINVAL, "m2c_residual_noalloc: stiffened-gas and Mie-Grueneisen materials only");
  // the EOS rules of m2c_set_eos: an unknown type or a parameter outside its
  // range is rejected before any device work
  if (const char* why = eos_desc_error(eos0))
    return noalloc_fail(M2C_EINVAL, std::string("m2c_residual_noalloc: material 0 EOS: ") + why);
  if (const char* why = eos_desc_error(eos1))
    return noalloc_fail(M2C_EINVAL, std::string("m2c_residual_noalloc: material 1 EOS: ") + why);
  const long long N = (long long)nx * ny * nz;
  if (N > m2c::kNoAllocMaxCells)
    return noalloc_fail(M2C_EINVAL, "m2c_residual_noalloc: " + std::to_string(N) + " cells exceed the maximum of " +
                                        std::to_string(m2c::kNoAllocMaxCells));
  void* base = nullptr;
  m2c_status st = noalloc_scratch(&base);
  if (st) return st;
  unsigned char* ws = static_cast<unsigned char*>(base);
  Grid g;
  std::memset(&g, 0, sizeof(g));
  g.nx = nx; g.ny = ny; g.nz = nz; g.N = N;
  for (int q = 0; q < 6; ++q) g.bc[q] = bc[q];
  g.active[0] = nx > 1; g.active[1] = ny > 1; g.active[2] = nz > 1;
  g.prec = precision;
  g.h = h; g.inv_h = 1.0 / h; g.cfl = 0.5;
  double p0[6], p1[6];
  for (int q = 0; q < 6; ++q) { p0[q] = eos0->params[q]; p1[q] = eos1->params[q]; }
  g.eos[0] = make_eos<double>(eos0->type, p0);
  g.eos[1] = make_eos<double>(eos1->type, p1);
  g.eosf[0] = make_eos<float>(eos0->type, p0);
  g.eosf[1] = make_eos<float>(eos1->type, p1);
  g.W = const_cast<double*>(W);
  g.phi = const_cast<double*>(phi);
  g.id = ws + m2c::kNaId;
  g.cell_slot = reinterpret_cast<int*>(ws + m2c::kNaSlot);
  g.faces = reinterpret_cast<IfFace*>(ws + m2c::kNaFaces);
  g.cells = reinterpret_cast<IfCell*>(ws + m2c::kNaCells);
  g.face_cap = (int)m2c::kNoAllocFaceCap;
  g.cell_cap = (int)m2c::kNoAllocCellCap;
  g.ctrl = reinterpret_cast<Ctrl*>(ws + m2c::kNaCtrl);
  g.resR = R;
  g.resL = L;
  const int ty = 8;
  set_tiling(g, ty, default_tz(g, ty));
  const long long tiles[2] = {0, ntiles_of(g)};
  Grid* dg = reinterpret_cast<Grid*>(ws + m2c::kNaGrid);
  long long* dt = reinterpret_cast<long long*>(ws + m2c::kNaTiles);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the previous call's contents stay in the array: reset the counters and the error latch
  cudaError_t e = cudaMemsetAsync(g.ctrl, 0, sizeof(Ctrl), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dg, &g, sizeof(Grid), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dt, tiles, sizeof(tiles), cudaMemcpyHostToDevice, s);
  LaunchPlan lp;
  lp.ty = ty;
  lp.mats = material_pair(g);
  if (e == cudaSuccess) e = launch_stage(precision, dg, dt, 1, tiles[1], kResidual, lp, s);
  if (e == cudaSuccess) {
    const dim3 lg((unsigned)(2 * sm_count()), 1);
    k_fiver<<<dim3((unsigned)(8 * sm_count()), 1), kFiverThreads, 0, s>>>(dg, kResidual);
    k_finish<<<lg, 128, 0, s>>>(dg, kResidual);
    e = cudaGetLastError();
  }
  Ctrl hc;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, g.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(M2C_ECUDA, std::string("m2c_residual_noalloc: ") + cudaGetErrorString(e));
  if (hc.err)
    return noalloc_fail((m2c_status)hc.err, std::string("m2c_residual_noalloc: device: ") +
                                                m2c_status_string(hc.err) + " at cell " + std::to_string(hc.err_cell));
  return M2C_OK;
}

m2c_status m2c_profile(m2c_ctx* c, int enable) {
  if (!c || enable < 0 || enable > 2) return M2C_EINVAL;
  c->profiling = enable != 0;
  c->profile_bulk_only = enable == 2;
  c->ev_used = 0;
  return M2C_OK;
}

m2c_status m2c_profile_read_kernels(m2c_ctx* c, double ms[6], long launches[6]) {
  if (!c || !ms || !launches) return M2C_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "profile_read");
  for (int k = 0; k < kKinds; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i < c->ev_used; ++i) {
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, c->ev[i].first, c->ev[i].second);
    if (e != cudaSuccess) return cuda_check(c, e, "profile_read");
    ms[c->ev_kind[i]] += t;
    launches[c->ev_kind[i]] += 1;
  }
  c->ev_used = 0;
  return M2C_OK;
}

m2c_status m2c_profile_read(m2c_ctx* c, double* total_ms, long* launches) {
  if (!c || !total_ms || !launches) return M2C_EINVAL;
  double ms[kKinds];
  long n[kKinds];
  m2c_status st = m2c_profile_read_kernels(c, ms, n);
  if (st) return st;
  *total_ms = ms[kKStage];
  *launches = n[kKStage];
  return M2C_OK;
}

void m2c_destroy(m2c_ctx* c) {
  if (!c) return;
  for (auto& p : c->ev) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  if (c->copy_in) {
    cudaStreamSynchronize(c->copy_in);
    for (int k = 0; k < 6; ++k) {
      if (c->down_ev[k]) cudaEventDestroy(c->down_ev[k]);
      if (c->up_ev[k]) cudaEventDestroy(c->up_ev[k]);
    }
    cudaStreamDestroy(c->copy_in);
  }
  delete c;
}

const char* m2c_last_error(const m2c_ctx* c) { return c ? c->err.c_str() : g_noctx_error.c_str(); }

}  // extern "C"
