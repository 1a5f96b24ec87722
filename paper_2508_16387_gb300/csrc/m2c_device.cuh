// Device helpers shared by the kernels of libm2cgpu: conservative to
// primitive conversion, face states, wave-speed sums and block reductions.
#pragma once
#include <cuda_runtime.h>

#include "m2c_kernels.cuh"

namespace m2c {

// Loads and stores of the state arrays as global-memory accesses: the pointers
// come from the grid descriptor, so the compiler cannot tell their address space
// and would otherwise use generic accesses. The loads go through the read-only
// path: within a launch no thread reads an address another thread writes (a
// stage reads one state and writes another; the last stage updates a cell in
// place after its own thread has read it).
__device__ __forceinline__ double gld(const double* p) { return __ldg(p); }
__device__ __forceinline__ void gst(double* p, double v) { __stwb(p, v); }

// ---------------------------------------------------------------------------
// Conservative -> primitive
// ---------------------------------------------------------------------------

// FP64 path: u = (rho u)/rho, e = (rho E - rho|V|^2/2)/rho, p = p(rho, e).
// Mixed path: the same with FP32 velocities and kinetic energy; rho e and, for
// the stiffened gas and NASG, the pressure (a difference of large numbers when
// p_c is large) in FP64, then rounded to FP32. EXT: NASG and JWL materials too;
// T: the material's type when fixed at compile time (-1: read from q).
//
// cons_to_prim_f is the mixed path after the loads: rho, rho u, rho v, rho w
// already rounded to binary32 (rf, f1, f2, f3), rho and rho E in binary64.
template <bool EXT = false, int T = -1>
__device__ __forceinline__ bool cons_to_prim_f(const EosP<float>& q, const EosDev& qd, double rho, float rf, float f1,
                                               float f2, float f3, double E, float P[5]) {
  const float inv = rrcp<float>(rf);
  const float u = f1 * inv, v = f2 * inv, w = f3 * inv;
  const float ke = 0.5f * ((f1 * u + f2 * v) + f3 * w);
  const double rhoe = E - f2d(ke);
  float p = 0.0f;
  bool ok = true;
  if (eos_is<T>(q, M2C_EOS_SG)) {
    p = d2f(qd.gm1 * rhoe - qd.gpc);
  } else if (EXT && eos_is<T>(q, M2C_EOS_NASG)) {
    const double d = 1.0 - rho * qd.b;
    ok = d > 0.0;
    p = d2f(div_nr(qd.gm1 * (rhoe - rho * qd.ec), d) - qd.gpc);
  } else {
    ok = eos_p<float, EXT, T>(q, rf, inv, d2f(rhoe) * inv, p);
  }
  P[0] = rf; P[1] = u; P[2] = v; P[3] = w; P[4] = p;
  return ok && gt0(rho);
}

template <typename R, bool EXT = false, int T = -1>
__device__ __forceinline__ bool cons_to_prim_v(const EosP<R>& q, const EosDev& qd, double rho, double m1, double m2,
                                               double m3, double E, R P[5]) {
  if constexpr (sizeof(R) == 8) {
    const double inv = rrcp<double>(rho);
    const double u = m1 * inv, v = m2 * inv, w = m3 * inv;
    const double ke = 0.5 * ((m1 * u + m2 * v) + m3 * w);
    const double e = (E - ke) * inv;
    double p = 0.0;
    const bool ok = eos_p<double, EXT, T>(q, rho, inv, e, p);
    P[0] = rho; P[1] = u; P[2] = v; P[3] = w; P[4] = p;
    return ok && rho > 0.0;
  } else {
    const double x[4] = {rho, m1, m2, m3};
    float y[4];
    d2f_group<4>(x, y);
    return cons_to_prim_f<EXT, T>(q, qd, rho, y[0], y[1], y[2], y[3], E, P);
  }
}

template <typename R, bool EXT = false>
__device__ __forceinline__ bool cons_to_prim(const EosP<R>& q, const EosDev& qd, const double* __restrict__ W,
                                             long long N, long long c, R P[5]) {
  return cons_to_prim_v<R, EXT>(q, qd, W[c], W[N + c], W[2 * N + c], W[3 * N + c], W[4 * N + c], P);
}

template <typename R, bool EXT = false, int T = -1>
__device__ __forceinline__ bool make_face(const EosP<R>& q, R rho, R u, R v, R w, R p, FaceState<R>& F) {
  R e = (R)0, c2 = (R)0;
  const bool ok = eos_e_c2<R, EXT, T>(q, rho, rrcp<R>(rho), p, e, c2);
  F.rho = rho; F.u = u; F.v = v; F.w = w; F.p = p;
  F.c = ok ? rsqrt_pos<R>(c2) : (R)0;
  F.E = e + (R)0.5 * ((u * u + v * v) + w * w);
  return ok;
}

// x == 0 (either sign), tested on the bits (off the FP64 pipe for FP64).
template <typename R>
__device__ __forceinline__ bool is_zero(R x) {
  if constexpr (sizeof(R) == 8) return ((hi_of(x) << 1) | lo_of(x)) == 0u;
  else return (bits_of(x) << 1) == 0u;
}

// MUSCL face states of one cell along one axis: q -+ sigma/2 with the modified
// van Albada slope (App. D). same = both stencil neighbours have the cell's
// material (otherwise first order, Reading R11); a non-admissible face state
// makes the whole axis first order (Reading R12). bad: even the cell state is
// not admissible. Where every slope vanishes (a locally uniform state) both
// face states are the cell state, which takes one EOS evaluation instead of two.
// The general kernels (GEN) take the limiter of the grid: lim = M2C_LIM_MC with
// alpha, else van Albada.
template <typename R, bool GEN = false, int T = -1>
__device__ __forceinline__ void cell_faces(const EosP<R>& q, const R Pm[5], const R P[5], const R Pp[5], bool same,
                                           FaceState<R>& Qm, FaceState<R>& Qp, bool& bad, int lim = 0,
                                           R alpha = (R)0) {
  if (same) {
    R s[5];
    if (GEN && lim == M2C_LIM_MC) {
#pragma unroll
      for (int v = 0; v < 5; ++v) s[v] = mc_slope<R>(P[v] - Pm[v], Pp[v] - P[v], alpha);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) s[v] = va_slope<R>(P[v] - Pm[v], Pp[v] - P[v]);
    }
    const bool flat = is_zero(s[0]) && is_zero(s[1]) && is_zero(s[2]) && is_zero(s[3]) && is_zero(s[4]);
    if (!flat) {
      const R hf = (R)0.5;
      const bool okm = make_face<R, GEN, T>(q, P[0] - hf * s[0], P[1] - hf * s[1], P[2] - hf * s[2],
                                            P[3] - hf * s[3], P[4] - hf * s[4], Qm);
      const bool okp = make_face<R, GEN, T>(q, P[0] + hf * s[0], P[1] + hf * s[1], P[2] + hf * s[2],
                                            P[3] + hf * s[3], P[4] + hf * s[4], Qp);
      if (okm && okp) return;
    }
  }
  if (!make_face<R, GEN, T>(q, P[0], P[1], P[2], P[3], P[4], Qm)) bad = true;
  Qp = Qm;
}

// Wave-speed sum of a state, sum over the axes with more than one cell of
// |V_d| + c (the CFL reading of the design notes), in precision R (the mixed
// path takes the time step from FP32 wave speeds of the FP64 state).
template <typename R, bool EXT = false, int T = -1>
__device__ __forceinline__ R wave_sum_v(const Grid& g, const EosP<R>& q, const EosDev& qd, const double w[5], bool& ok) {
  R P[5];
  ok = cons_to_prim_v<R, EXT, T>(q, qd, w[0], w[1], w[2], w[3], w[4], P);
  R e, c2;
  ok = ok && eos_e_c2<R, EXT, T>(q, P[0], rrcp<R>(P[0]), P[4], e, c2);
  const R cs = ok ? rsqrt_pos<R>(c2) : (R)0;
  R lam = (R)0;
  if (g.active[0]) lam = lam + (fabs(P[1]) + cs);
  if (g.active[1]) lam = lam + (fabs(P[2]) + cs);
  if (g.active[2]) lam = lam + (fabs(P[3]) + cs);
  return lam;
}

template <typename R>
__device__ __forceinline__ double wave_sum_r(const Grid& g, const EosP<R>& q, const EosDev& qd, const double* W,
                                             long long N, long long c, bool& ok) {
  const double w[5] = {W[c], W[N + c], W[2 * N + c], W[3 * N + c], W[4 * N + c]};
  return to_d<R>(wave_sum_v<R, true>(g, q, qd, w, ok));
}

// The same in the grid's precision, for material m: every wave-speed maximum
// of a grid (first step, bulk, interface and flipped cells) is taken the same
// way, so that a step from a restored state repeats the uninterrupted one.
__device__ __forceinline__ double wave_sum(const Grid& g, int m, const double* W, long long N, long long c,
                                           bool& ok) {
  if (g.prec == M2C_MIXED) return wave_sum_r<float>(g, g.eosf[m], g.eos[m], W, N, c, ok);
  return wave_sum_r<double>(g, g.eos[m], g.eos[m], W, N, c, ok);
}

// Narrow-band level set (Sec. 4.4; the local level set of Peng et al., J.
// Comput. Phys. 155, 1999): the advection velocity is scaled by
// c = 1 for |phi| <= beta, (|phi| - gamma)^2 (2|phi| + gamma - 3 beta)/(gamma - beta)^3
// between the tube radii, 0 beyond gamma.
template <typename R>
__device__ __forceinline__ R band_cutoff(R beta, R gamma, R phi) {
  const R a = fabs(phi);
  if (a <= beta) return (R)1;
  if (a >= gamma) return (R)0;
  const R d = gamma - beta, x = a - gamma;
  return rdiv<R>(x * x * ((R)2 * a + gamma - (R)3 * beta), d * d * d);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block max of a positive double, then one atomic max on its bit pattern
// (positive doubles order like their bit patterns).
__device__ __forceinline__ void block_max_to(double v, unsigned long long* dst, double* s_red) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) s_red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double x = lane < nw ? s_red[lane] : 0.0;
    x = warp_max(x);
    if (lane == 0 && x > 0.0) atomicMax(dst, (unsigned long long)__double_as_longlong(x));
  }
}

__device__ __forceinline__ int find_grid(const long long* __restrict__ tile_begin, int ngrid, long long tile) {
  int lo = 0, hi = ngrid - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_begin[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace m2c
