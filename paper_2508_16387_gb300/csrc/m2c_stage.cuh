// The bulk stage kernel k_stage<R, TY> (a template instantiated per precision
// in m2c_stage_fp32.cu and m2c_stage_fp64.cu) and its launch helpers.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "m2c_device.cuh"
#include "m2c_stage.h"

namespace m2c {

// ---------------------------------------------------------------------------
// Bulk stage kernel
// ---------------------------------------------------------------------------

// The level set and material planes are double-buffered where shared memory
// allows (16-row FP32 tiles at two blocks per SM, FP64 tiles at one): a plane's
// update reads them while the next plane's loads already write the other
// buffer, which saves one block barrier per plane. The 8-row FP32 tiles (four
// blocks per SM) keep one buffer and the barrier.
template <typename R, int TY>
struct StageSmem {
  static constexpr int TX = 32, HX = TX + 4, HY = TY + 4;
  static constexpr int NB = (TY >= 16 || sizeof(R) == 8) ? 2 : 1;
  static constexpr size_t q_off = 0;
  static constexpr size_t phi_off = q_off + sizeof(R) * 5 * HY * HX;
  static constexpr size_t xs_off = phi_off + sizeof(R) * NB * HY * HX;
  static constexpr size_t ys_off = xs_off + sizeof(FaceState<R>) * TY * (TX + 2) * 2;
  static constexpr size_t fx_off = ys_off + sizeof(FaceState<R>) * (TY + 2) * TX * 2;
  static constexpr size_t fy_off = fx_off + sizeof(R) * 5 * TY * (TX + 1);
  static constexpr size_t id_off = fy_off + sizeof(R) * 5 * (TY + 1) * TX;
  static constexpr size_t bytes = (id_off + NB * HY * HX + 15) / 16 * 16;
};

// Compile-time integer for the material dispatch below (usable in device code).
template <int V>
struct IntC {
  static constexpr int value = V;
  __device__ constexpr operator int() const { return V; }
};

// Calls f(T, m) for material m of a cell: T its EOS type as a compile-time
// constant when the instantiation fixes the pair of material types (MT = T0 +
// 4 T1, each M2C_EOS_SG or M2C_EOS_MG), else IntC<-1> (the type is read at run
// time); m the material index, itself a compile-time constant where the two
// fixed types differ (f is then inlined once per material).
template <int MT, typename F>
__device__ __forceinline__ void by_material(int m, F&& f) {
  if constexpr (MT < 0) {
    f(IntC<-1>{}, m);
  } else if constexpr ((MT & 3) == (MT >> 2)) {
    f(IntC<(MT & 3)>{}, m);
  } else {
    if (m == 0) f(IntC<(MT & 3)>{}, IntC<0>{});
    else f(IntC<(MT >> 2)>{}, IntC<1>{});
  }
}

// FP64 tiles run one block per SM (FP64-pipe bound); the FP32 tiles of the
// mixed path are latency bound and are compiled for 1024 resident threads per
// SM (64 registers a thread): four 256-thread blocks of 8-row tiles (55 KB of
// shared memory each) or two 512-thread blocks of 16-row tiles.
//
// Every thread's share of the plane work (halo cell, face-state items, flux
// items) and its shared-memory addresses are fixed for the whole launch; only
// the plane index changes along the march. The halo slots are computed once,
// the face-state and flux items are recomputed from the thread index where
// they are used (cheaper than holding them in registers across the march).
//
// GEN = false is the default scheme (TVD RK2, modified van Albada, HLLC); GEN =
// true is the general instantiation, which takes the grid's scheme options at
// run time (limiter, flux, the stages of TVD RK3) at some cost in registers.
// MT >= 0 fixes the EOS types of the two materials (SG or MG, MT = T0 + 4 T1)
// for launches whose grids all have that pair, which removes the type dispatch
// from every EOS evaluation; MT = -1 reads the types at run time.
template <typename R, int TY, bool GEN, int MT = -1>
__global__ void __launch_bounds__(32 * TY, (sizeof(R) == 8 ? 1 : 1024 / (32 * TY)))
k_stage(const Grid* __restrict__ grids, const long long* __restrict__ tile_begin, int ngrid, long long ntiles, int mode,
        int sched, unsigned long long* __restrict__ tile_counter) {
  constexpr int TX = 32, NT = TX * TY, HX = TX + 4, HY = TY + 4, PL = HY * HX;
  constexpr int NXS = (TX + 2) * TY, NYS = TX * (TY + 2), NS = NXS + NYS;  // face-state items
  constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1), NF = NXF + NYF;  // flux items
  constexpr int NHALO = 4 * (TX + TY);
  constexpr int SI = (NS + NT - 1) / NT, FI = (NF + NT - 1) / NT;
  constexpr int SFX = TY * (TX + 1), SFY = (TY + 1) * TX;                   // flux array strides
  using SM = StageSmem<R, TY>;
  extern __shared__ __align__(16) unsigned char smem[];
  R* s_q = reinterpret_cast<R*>(smem + SM::q_off);                         // [5][HY][HX]
  R* const s_phi0 = reinterpret_cast<R*>(smem + SM::phi_off);               // [NB][HY][HX]
  FaceState<R>* s_st = reinterpret_cast<FaceState<R>*>(smem + SM::xs_off);  // x: [TY][TX+2][2], then y: [TY+2][TX][2]
  R* s_fx = reinterpret_cast<R*>(smem + SM::fx_off);                       // [5][TY][TX+1]
  R* s_fy = reinterpret_cast<R*>(smem + SM::fy_off);                       // [5][TY+1][TX]
  uint8_t* const s_id0 = smem + SM::id_off;                                // [NB][HY][HX]
  // the descriptor of the tile's grid, copied to shared memory for each tile
  // (its fields and EOS parameters are read all through the plane loop)
  __shared__ __align__(16) Grid s_G;
  static_assert(sizeof(Grid) % 8 == 0, "grid descriptor copy");
  const EosP<R>* s_eos;
  if constexpr (sizeof(R) == 8) s_eos = s_G.eos;
  else s_eos = s_G.eosf;
  const EosDev* s_eosd = s_G.eos;
  __shared__ double s_dt;
  __shared__ double s_red[32];
  __shared__ long long s_tile;

  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const unsigned lane = tid & 31, lt = (1u << lane) - 1u;

  // The thread's share of the plane work is recomputed from the thread index
  // where it is used (a volatile read of %tid.x keeps the compiler from
  // holding the items in registers across the plane loop).
  auto tid_now = []() {
    unsigned t;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
    return (int)t;
  };
  // face-state item s, packed: centre in the plane buffer (bits 0-9), stencil along y (bit 10); -1: none
  auto st_item = [&](int s) {
    const int i = tid_now() + s * NT;
    if (i < NXS) return (i / (TX + 2) + 2) * HX + i % (TX + 2) + 1;
    if (i < NS) {
      const int j = i - NXS;
      return ((j / TX + 1) * HX + j % TX + 2) | (1 << 10);
    }
    return -1;
  };
  // flux item s, packed in two words: left face state (bits 0-15) and direction y (bit 30),
  // -1: none; id position of the left cell (bits 0-15) and output offset (bits 16-31)
  auto flux_item = [&](int s, int& b) {
    const int i = tid_now() + s * NT;
    if (i < NXF) {
      const int f = i % (TX + 1), row = i / (TX + 1);
      b = ((row + 2) * HX + f + 1) | ((row * (TX + 1) + f) << 16);
      return 2 * (row * (TX + 2) + f) + 1;
    }
    if (i < NF) {
      const int j = i - NXF;
      const int x = j % TX, f = j / TX;
      b = ((f + 1) * HX + x + 2) | ((f * TX + x) << 16);
      return (2 * NXS + 2 * (f * TX + x) + 1) | (1 << 30);
    }
    b = 0;
    return -1;
  };
  static_assert(2 * NS < 65536 && PL < 1024 && SFX < 32768 && SFY < 32768, "packed item fields");
  // halo cells of the plane buffer loaded by this thread (two-cell ring without corners):
  // smem slot, or -1
  constexpr int HI = (NHALO + NT - 1) / NT;
  int h_hx[HI], h_hy[HI];
#pragma unroll
  for (int s = 0; s < HI; ++s) {
    const int h = tid + s * NT;
    h_hx[s] = -1;
    h_hy[s] = 0;
    if (h < 4 * TY) {
      const int c4 = h / TY;
      h_hx[s] = c4 < 2 ? c4 : TX + c4;
      h_hy[s] = h % TY + 2;
    } else if (h < NHALO) {
      const int h2 = h - 4 * TY;
      const int c4 = h2 / TX;
      h_hy[s] = c4 < 2 ? c4 : TY + c4;
      h_hx[s] = h2 % TX + 2;
    }
  }

  // Tiles of all grids of the launch, taken in order by a fixed stride
  // (sched 0) or from an atomic counter (sched 1).
  for (long long iter = 0;; ++iter) {
  long long tile;
  if (sched == 1) {
    if (tid == 0) s_tile = (long long)atomicAdd(tile_counter, 1ull);
    __syncthreads();
    tile = s_tile;
  } else {
    tile = blockIdx.x + iter * (long long)gridDim.x;
  }
  if (tile >= ntiles) break;
  const int gidx = find_grid(tile_begin, ngrid, tile);
  {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(grids + gidx);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_G);
    for (int i = tid; i < (int)(sizeof(Grid) / 8); i += NT) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  const Grid& G = s_G;
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const long long N = G.N, nxy = (long long)nx * ny;
  const int bcz0 = G.bc[4], bcz1 = G.bc[5];
  long long t = tile - tile_begin[gidx];
  const int bx = (int)(t % G.tiles_x);
  t /= G.tiles_x;
  const int by = (int)(t % G.tiles_y);
  const int bz = (int)(t / G.tiles_y);
  const int x0 = bx * TX, y0 = by * TY, k0 = bz * G.tz, k1 = min(k0 + G.tz, nz);
  const R ih = (R)G.inv_h;
  const R i6h = (R)(1.0 / (6.0 * G.h));
  const double* __restrict__ Ws = GEN ? stage_W(G, mode) : (mode == kStage2 ? G.W1 : G.W);
  const double* __restrict__ phis = GEN ? stage_phi(G, mode) : (mode == kStage2 ? G.phi1 : G.phi);
  const uint8_t* __restrict__ idg = G.id;
  Ctrl* ctrl = G.ctrl;
  const int slot = GEN ? list_slot(mode) : (mode == kStage2 ? 1 : 0);
  // material ids are frozen after the first stage of a step
  const bool ids_frozen = GEN ? (mode != kStage1 && mode != kResidual) : mode == kStage2;
  const bool final_stage = GEN ? last_stage(mode) : mode == kStage2;
  const int lim = GEN ? G.limiter : 0, flx = GEN ? G.flux : 0;
  const R alpha = GEN ? (R)G.mc_alpha : (R)0;
  const long long step = ctrl->step;

  if (tid == 0) s_dt = mode == kResidual ? 0.0 : lam_to_dt(G, ctrl->lam[step & 1]);
  __syncthreads();
  const double dt = s_dt;
  const R hdt = to_r<R>(0.5 * dt);

  const int gx = x0 + tx, gy = y0 + ty;
  const bool inside = gx < nx && gy < ny;
  // column bases (x, y mapped once per tile)
  const long long own_base = (long long)map_index(gy, ny, G.bc[2], G.bc[3]) * nx + map_index(gx, nx, G.bc[0], G.bc[1]);
  long long halo_base[HI];
#pragma unroll
  for (int s = 0; s < HI; ++s)
    halo_base[s] = h_hx[s] < 0 ? 0
                               : (long long)map_index(y0 + h_hy[s] - 2, ny, G.bc[2], G.bc[3]) * nx +
                                     map_index(x0 + h_hx[s] - 2, nx, G.bc[0], G.bc[1]);
  // general kernel: velocity components to negate for a position mirrored across a
  // symmetry side (bit 0: u, bit 1: v, bit 2: w), for the own column and the halo slots
  int own_neg = 0, halo_neg[HI];
#pragma unroll
  for (int s = 0; s < HI; ++s) halo_neg[s] = 0;
  if constexpr (GEN) {
    own_neg = mirrored(gx, nx, G.bc[0], G.bc[1]) | (mirrored(gy, ny, G.bc[2], G.bc[3]) << 1);
#pragma unroll
    for (int s = 0; s < HI; ++s)
      if (h_hx[s] >= 0)
        halo_neg[s] = mirrored(x0 + h_hx[s] - 2, nx, G.bc[0], G.bc[1]) |
                      (mirrored(y0 + h_hy[s] - 2, ny, G.bc[2], G.bc[3]) << 1);
  }
  auto zneg = [&](int k) { return GEN ? (mirrored(k, nz, bcz0, bcz1) << 2) : 0; };

  // failures seen by this thread in this tile: non-physical state, work-list overflow
  bool bad = false, ovf = false;
  // material at the start of the step and the stage state of cell index c
  // (neg: the velocity components to negate, general kernel only)
  auto load = [&](long long c, R P[5], R& ph, int& idv, int neg) {
    const double phd = gld(phis + c);
    if (ids_frozen) {
      idv = __ldg(idg + c) & 1;
    } else {
      idv = lt0(phd) ? 1 : 0;
    }
    const double w0 = gld(Ws + c), w1 = gld(Ws + N + c), w2 = gld(Ws + 2 * N + c), w3 = gld(Ws + 3 * N + c),
                 w4 = gld(Ws + 4 * N + c);
    if constexpr (sizeof(R) == 8) {
      ph = phd;
      by_material<MT>(idv, [&](auto T, auto m) {
        if (!cons_to_prim_v<R, GEN, decltype(T)::value>(s_eos[m], s_eosd[m], w0, w1, w2, w3, w4, P)) bad = true;
      });
    } else {
      // the level set and the state's first four components: one group of conversions
      const double x[5] = {phd, w0, w1, w2, w3};
      float y[5];
      d2f_group<5>(x, y);
      ph = y[0];
      by_material<MT>(idv, [&](auto T, auto m) {
        if (!cons_to_prim_f<GEN, decltype(T)::value>(s_eos[m], s_eosd[m], w0, y[1], y[2], y[3], y[4], w4, P))
          bad = true;
      });
    }
    if constexpr (GEN) {
      if (neg & 1) P[1] = -P[1];
      if (neg & 2) P[2] = -P[2];
      if (neg & 4) P[3] = -P[3];
    }
  };
  auto plane = [&](int k) { return (long long)map_index(k, nz, bcz0, bcz1) * nxy; };

  // ---- warm-up of the z window: planes k0-2 .. k0+1
  R Pa[5], P0[5], P1[5], P2[5];
  R ph[5];
  int ida, idm, id0, id1, id2;
  FaceState<R> QzP, Qtmp, QzM1, QzP1;
  R Fzm[5], Fzp[5];
  {
    R Pb[5];
    int idb;
    load(plane(k0 - 2) + own_base, Pb, ph[0], idb, own_neg | zneg(k0 - 2));
    load(plane(k0 - 1) + own_base, Pa, ph[1], ida, own_neg | zneg(k0 - 1));
    load(plane(k0) + own_base, P0, ph[2], id0, own_neg);
    load(plane(k0 + 1) + own_base, P1, ph[3], id1, own_neg | zneg(k0 + 1));
    FaceState<R> QaP, Q0M;
    by_material<MT>(ida, [&](auto T, auto m) {
      cell_faces<R, GEN, decltype(T)::value>(s_eos[m], Pb, Pa, P0, idb == ida && id0 == ida, Qtmp, QaP, bad, lim,
                                              alpha);
    });
    by_material<MT>(id0, [&](auto T, auto m) {
      cell_faces<R, GEN, decltype(T)::value>(s_eos[m], Pa, P0, P1, ida == id0 && id1 == id0, Q0M, QzP, bad, lim,
                                              alpha);
    });
    if (ida == id0) {
      num_flux<2, R, GEN>(QaP, Q0M, Fzm, flx);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) Fzm[v] = (R)0;
    }
    idm = ida;
  }

  R lam_max = (R)0;
  const int cslot = (ty + 2) * HX + tx + 2;

  for (int k = k0; k < k1; ++k) {
    const long long pk = (long long)k * nxy;  // k is inside the grid
    const int buf = SM::NB == 2 ? ((k - k0) & 1) : 0;
    R* const s_phi = s_phi0 + buf * PL;
    uint8_t* const s_id = s_id0 + buf * PL;
    // ---- own column: plane k+2, z face states of cell k+1, z flux of face k+1/2
    load(plane(k + 2) + own_base, P2, ph[4], id2, own_neg | zneg(k + 2));
    by_material<MT>(id1, [&](auto T, auto m) {
      cell_faces<R, GEN, decltype(T)::value>(s_eos[m], P0, P1, P2, id0 == id1 && id2 == id1, QzM1, QzP1, bad, lim,
                                              alpha);
    });
    if (id0 == id1) {
      num_flux<2, R, GEN>(QzP, QzM1, Fzp, flx);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) Fzp[v] = (R)0;
    }
    // ---- plane k into shared memory: own cells and the two-cell halo (no corners)
#pragma unroll
    for (int v = 0; v < 5; ++v) s_q[v * PL + cslot] = P0[v];
    s_phi[cslot] = ph[2];
    s_id[cslot] = (uint8_t)id0;
#pragma unroll
    for (int s = 0; s < HI; ++s) {
      if (h_hx[s] < 0) break;
      const int hslot = h_hy[s] * HX + h_hx[s];
      R Ph[5], phh;
      int idh;
      load(pk + halo_base[s], Ph, phh, idh, halo_neg[s]);
#pragma unroll
      for (int v = 0; v < 5; ++v) s_q[v * PL + hslot] = Ph[v];
      s_phi[hslot] = phh;
      s_id[hslot] = (uint8_t)idh;
    }
    __syncthreads();

    // ---- MUSCL face states along x (cells x = -1 .. TX) and y (cells y = -1 .. TY)
#pragma unroll
    for (int s = 0; s < SI; ++s) {
      const int it = st_item(s);
      if (it < 0) break;
      const int c0 = it & 1023, so = (it >> 10) ? HX : 1;
      R Pm[5], P[5], Pp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Pm[v] = s_q[v * PL + c0 - so];
        P[v] = s_q[v * PL + c0];
        Pp[v] = s_q[v * PL + c0 + so];
      }
      const int ic = s_id[c0];
      const bool same = s_id[c0 - so] == ic && s_id[c0 + so] == ic;
      bool b = false;
      FaceState<R>* out = s_st + 2 * (tid + s * NT);
      by_material<MT>(ic, [&](auto T, auto m) {
        cell_faces<R, GEN, decltype(T)::value>(s_eos[m], Pm, P, Pp, same, out[0], out[1], b, lim, alpha);
      });
      bad = bad || b;
    }
    __syncthreads();

    // ---- HLLC on every x face (between cells f-1 and f of a row) and y face of the tile
#pragma unroll
    for (int s = 0; s < FI; ++s) {
      int itb;
      const int it = flux_item(s, itb);
      if (it < 0) break;
      const int dir = (it >> 30) & 1;
      const int lsi = it & 0xffff, idp = itb & 0xffff, outo = (itb >> 16) & 0x7fff;
      const int il = s_id[idp], ir = s_id[idp + (dir ? HX : 1)];
      const FaceState<R>& QL = s_st[lsi];
      const FaceState<R>& QR = s_st[lsi + (dir ? 2 * TX - 1 : 1)];
      R F[5];
      if (il != ir) {
#pragma unroll
        for (int v = 0; v < 5; ++v) F[v] = (R)0;
      } else if (dir == 0) {
        num_flux<0, R, GEN>(QL, QR, F, flx);
      } else {
        num_flux<1, R, GEN>(QL, QR, F, flx);
      }
      R* o = (dir ? s_fy : s_fx) + outo;
      const int stride = dir ? SFY : SFX;
#pragma unroll
      for (int v = 0; v < 5; ++v) o[v * stride] = F[v];
    }
    __syncthreads();

    // ---- per cell: residual, level set, Runge-Kutta update, work lists
    {
      const int idxm = s_id[cslot - 1], idxp = s_id[cslot + 1];
      const int idym = s_id[cslot - HX], idyp = s_id[cslot + HX];
      const bool is_if = inside && (idxm != id0 || idxp != id0 || idym != id0 || idyp != id0 || idm != id0 ||
                                    id1 != id0);
      R res[5];
      R Fxm[5], Fxp[5], Fym[5], Fyp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Fxm[v] = s_fx[v * SFX + ty * (TX + 1) + tx];
        Fxp[v] = s_fx[v * SFX + ty * (TX + 1) + tx + 1];
        Fym[v] = s_fy[v * SFY + ty * TX + tx];
        Fyp[v] = s_fy[v * SFY + (ty + 1) * TX + tx];
        res[v] = ((Fxm[v] - Fxp[v]) * ih + (Fym[v] - Fyp[v]) * ih) + (Fzm[v] - Fzp[v]) * ih;
      }
      // level-set residual -((u phi_x + v phi_y) + w phi_z), third-order upwind-biased (Sec. 4.4)
      const R u = P0[1], vv = P0[2], w = P0[3];
      const R* prow = s_phi + cslot;
      R Dx, Dy, Dz;
      if (u >= (R)0) Dx = (((R)2 * prow[1] + (R)3 * prow[0]) - (R)6 * prow[-1] + prow[-2]) * i6h;
      else Dx = ((-prow[2] + (R)6 * prow[1]) - (R)3 * prow[0] - (R)2 * prow[-1]) * i6h;
      if (vv >= (R)0) Dy = (((R)2 * prow[HX] + (R)3 * prow[0]) - (R)6 * prow[-HX] + prow[-2 * HX]) * i6h;
      else Dy = ((-prow[2 * HX] + (R)6 * prow[HX]) - (R)3 * prow[0] - (R)2 * prow[-HX]) * i6h;
      if (w >= (R)0) Dz = (((R)2 * ph[3] + (R)3 * ph[2]) - (R)6 * ph[1] + ph[0]) * i6h;
      else Dz = ((-ph[4] + (R)6 * ph[3]) - (R)3 * ph[2] - (R)2 * ph[1]) * i6h;
      R Lphi = -((u * Dx + vv * Dy) + w * Dz);
      if constexpr (GEN) {
        // narrow band (Sec. 4.4): the velocity scaled by the cutoff of the cell's level set
        if (G.band_gamma > 0.0) Lphi = band_cutoff<R>((R)G.band_beta, (R)G.band_gamma, ph[2]) * Lphi;
      }

      const long long c = pk + own_base;
      if constexpr (GEN) {
        // spherical / cylindrical forms (Sec. 3.4): S = -(alpha/r) u_r (rho, rho u, rho v,
        // rho w, rho E + p) at the cell centre r = x0 + (i + 1/2) h from the stage state,
        // added after the flux sum (interface cells get it in k_finish)
        if (G.geom != M2C_GEOM_CARTESIAN && inside && !is_if) {
          const double r = G.x0 + ((double)gx + 0.5) * G.h;
          const R a = to_r<R>((G.geom == M2C_GEOM_SPHERICAL ? 2.0 : 1.0) / r) * P0[1];
          R wv[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) wv[v] = to_r<R>(gld(Ws + v * N + c));
#pragma unroll
          for (int v = 0; v < 4; ++v) res[v] = res[v] - a * wv[v];
          res[4] = res[4] - a * (wv[4] + P0[4]);
        }
      }
      bool flip = false;
      if (inside) {
        if (mode == kResidual) {
          if (!is_if) {
#pragma unroll
            for (int v = 0; v < 5; ++v) G.resR[v * N + c] = to_d<R>(res[v]);
          }
          G.resL[c] = to_d<R>(Lphi);
          G.id[c] = (uint8_t)id0;
        } else if (mode == kStage1) {
          gst(G.phi1 + c, gld(G.phi + c) + dt * to_d<R>(Lphi));
          G.id[c] = (uint8_t)id0;
          if (!is_if) {
#pragma unroll
            for (int v = 0; v < 5; ++v) gst(G.W1 + v * N + c, gld(G.W + v * N + c) + dt * to_d<R>(res[v]));
          }
        } else if (GEN && mode == kStage2of3) {
          // TVD RK3, second stage (Sec. 4.3): W2 = (3/4 W + 1/4 W1) + 1/4 dt R(W1)
          gst(G.phi2 + c, (0.75 * gld(G.phi + c) + 0.25 * gld(G.phi1 + c)) + 0.25 * dt * to_d<R>(Lphi));
          if (!is_if) {
#pragma unroll
            for (int v = 0; v < 5; ++v)
              gst(G.W2 + v * N + c,
                  (0.75 * gld(G.W + v * N + c) + 0.25 * gld(G.W1 + v * N + c)) + 0.25 * dt * to_d<R>(res[v]));
          }
        } else {
          // last stage: TVD RK2 W' = (W + (W1 + dt R(W1)))/2, or TVD RK3
          // W' = (1/3 W + 2/3 W2) + 2/3 dt R(W2). The mixed path's TVD RK2 takes
          // W' = (W + W1)/2 + (dt/2) R with the increment (dt/2) R in binary32 (R
          // itself is a binary32 result) and one rounding after the FP64 sum.
          const bool rk3 = GEN && mode == kStage3;
          constexpr bool f32inc = sizeof(R) == 4 && !GEN;
          const double pn = rk3      ? (gld(G.phi + c) / 3.0 + 2.0 / 3.0 * gld(G.phi2 + c)) +
                                      2.0 / 3.0 * dt * to_d<R>(Lphi)
                            : f32inc ? fma(0.5, gld(G.phi + c) + gld(G.phi1 + c), to_d<R>(hdt * Lphi))
                                     : 0.5 * (gld(G.phi + c) + (gld(G.phi1 + c) + dt * to_d<R>(Lphi)));
          gst(G.phi + c, pn);
          const bool neg = lt0(pn);
          flip = neg != (id0 == 1);
          // bit 2: material at the end of the step (read by the phase update)
          G.id[c] = (uint8_t)(id0 | (neg ? 4 : 0));
          if (!is_if) {
            double wn[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              wn[v] = rk3      ? (gld(G.W + v * N + c) / 3.0 + 2.0 / 3.0 * gld(G.W2 + v * N + c)) +
                                2.0 / 3.0 * dt * to_d<R>(res[v])
                      : f32inc ? fma(0.5, gld(G.W + v * N + c) + gld(G.W1 + v * N + c), to_d<R>(hdt * res[v]))
                               : 0.5 * (gld(G.W + v * N + c) + (gld(G.W1 + v * N + c) + dt * to_d<R>(res[v])));
              gst(G.W + v * N + c, wn[v]);
            }
            if (!flip) {
              bool ok;
              R lam = (R)0;
              by_material<MT>(id0, [&](auto T, auto m) {
                lam = wave_sum_v<R, GEN, decltype(T)::value>(G, s_eos[m], s_eosd[m], wn, ok);
              });
              bad = bad || !ok;
              lam_max = fmax(lam_max, lam);
            }
          }
        }
      }
      // ---- work lists: warp ballot, one atomic per warp (skipped when the warp has none)
      const bool fxf = inside && idxp != id0, fyf = inside && idyp != id0, fzf = inside && id1 != id0;
      const int nf = (int)fxf + (int)fyf + (int)fzf;
      if (__any_sync(0xffffffffu, is_if || nf || flip)) {
        {
          const unsigned m = __ballot_sync(0xffffffffu, is_if);
          if (m) {
            int base = 0;
            const int leader = __ffs(m) - 1;
            if ((int)lane == leader) base = atomicAdd(&ctrl->ncell[slot], __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (is_if) {
              const int s = base + __popc(m & lt);
              if (s < G.cell_cap) {
                IfCell* e = G.cells + s;
                e->cell = c;
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                  e->F[0][v] = to_d<R>(Fxm[v]);
                  e->F[1][v] = to_d<R>(Fxp[v]);
                  e->F[2][v] = to_d<R>(Fym[v]);
                  e->F[3][v] = to_d<R>(Fyp[v]);
                  e->F[4][v] = to_d<R>(Fzm[v]);
                  e->F[5][v] = to_d<R>(Fzp[v]);
                }
                G.cell_slot[c] = s;
              } else {
                ovf = true;
              }
            }
          }
        }
        {
          int incl = nf;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += y;
          }
          const int total = __shfl_sync(0xffffffffu, incl, 31);
          if (total) {
            int base = 0;
            if (lane == 31) base = atomicAdd(&ctrl->nface[slot], total);
            base = __shfl_sync(0xffffffffu, base, 31);
            int s = base + incl - nf;
            const bool fl[3] = {fxf, fyf, fzf};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              if (fl[d]) {
                if (s < G.face_cap) {
                  G.faces[s].cell = c;
                  G.faces[s].dir = d;
                } else {
                  ovf = true;
                }
                ++s;
              }
            }
          }
        }
        if (final_stage) {
          const unsigned m = __ballot_sync(0xffffffffu, flip);
          if (m) {
            int base = 0;
            const int leader = __ffs(m) - 1;
            if ((int)lane == leader) base = atomicAdd(&ctrl->nflip, __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (flip) {
              const int s = base + __popc(m & lt);
              if (s < G.flip_cap) G.flips[s] = c;
              else ovf = true;
            }
          }
        }
      }
    }
    if constexpr (SM::NB == 1) __syncthreads();  // the next plane overwrites s_phi and s_id

    // ---- shift the z window
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      P0[v] = P1[v];
      P1[v] = P2[v];
      Fzm[v] = Fzp[v];
    }
    ph[0] = ph[1]; ph[1] = ph[2]; ph[2] = ph[3]; ph[3] = ph[4];
    idm = id0; id0 = id1; id1 = id2;
    QzP = QzP1;
  }
  // failures are latched once per tile, with the thread's column at the tile's first plane
  if (bad) latch_error(ctrl, M2C_ENONPHYS, cell_of(G, gx, gy, k0));
  if (ovf) latch_error(ctrl, M2C_EOVERFLOW, cell_of(G, gx, gy, k0));
  if (final_stage) block_max_to(to_d<R>(lam_max), &ctrl->lam[(step + 1) & 1], s_red);
  __syncthreads();  // the next tile reuses the shared memory
  }
}

// The shared-memory opt-in is a per-device attribute of the kernel: it is set
// once on every device the calling threads make current.
template <typename R, int TY, bool GEN, int MT = -1>
void stage_smem_setup() {
  static bool done[kMaxDevices] = {};
  const int dev = current_device();
  if (done[dev]) return;
  cudaFuncSetAttribute(k_stage<R, TY, GEN, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)StageSmem<R, TY>::bytes);
  done[dev] = true;
}

template <typename R, int TY, bool GEN, int MT = -1>
cudaError_t launch_stage_t(const Grid* grids, const long long* tiles, int ngrid, long long ntiles, int mode,
                           const LaunchPlan& lp, cudaStream_t s) {
  stage_smem_setup<R, TY, GEN, MT>();
  long long nb = ntiles;
  if (lp.blocks_per_sm > 0) nb = std::min<long long>(ntiles, (long long)lp.blocks_per_sm * sm_count());
  if (nb < 1) nb = 1;
  if (lp.sched == 1) {
    cudaError_t e = cudaMemsetAsync(lp.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  k_stage<R, TY, GEN, MT><<<(unsigned)nb, 32 * TY, StageSmem<R, TY>::bytes, s>>>(grids, tiles, ngrid, ntiles, mode,
                                                                              lp.sched, lp.counter);
  return cudaGetLastError();
}

// The launch for the material pair of the plan: instantiations with fixed EOS
// types for the four SG / MG pairs, else the run-time types.
template <typename R, int TY>
cudaError_t launch_stage_pair(const Grid* grids, const long long* tiles, int ngrid, long long ntiles, int mode,
                              const LaunchPlan& lp, cudaStream_t s) {
  switch (lp.mats) {
    case M2C_EOS_SG + 4 * M2C_EOS_SG:
      return launch_stage_t<R, TY, false, M2C_EOS_SG + 4 * M2C_EOS_SG>(grids, tiles, ngrid, ntiles, mode, lp, s);
    case M2C_EOS_MG + 4 * M2C_EOS_SG:
      return launch_stage_t<R, TY, false, M2C_EOS_MG + 4 * M2C_EOS_SG>(grids, tiles, ngrid, ntiles, mode, lp, s);
    case M2C_EOS_SG + 4 * M2C_EOS_MG:
      return launch_stage_t<R, TY, false, M2C_EOS_SG + 4 * M2C_EOS_MG>(grids, tiles, ngrid, ntiles, mode, lp, s);
    case M2C_EOS_MG + 4 * M2C_EOS_MG:
      return launch_stage_t<R, TY, false, M2C_EOS_MG + 4 * M2C_EOS_MG>(grids, tiles, ngrid, ntiles, mode, lp, s);
    default:
      return launch_stage_t<R, TY, false>(grids, tiles, ngrid, ntiles, mode, lp, s);
  }
}

template <typename R, int TY>
void stage_smem_setup_pairs() {
  stage_smem_setup<R, TY, false, M2C_EOS_SG + 4 * M2C_EOS_SG>();
  stage_smem_setup<R, TY, false, M2C_EOS_MG + 4 * M2C_EOS_SG>();
  stage_smem_setup<R, TY, false, M2C_EOS_SG + 4 * M2C_EOS_MG>();
  stage_smem_setup<R, TY, false, M2C_EOS_MG + 4 * M2C_EOS_MG>();
  stage_smem_setup<R, TY, false>();
}

}  // namespace m2c
