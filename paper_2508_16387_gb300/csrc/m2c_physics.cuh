// Device-side physics of the M2C finite-volume step (arXiv 2508.16387):
// equations of state, the modified van Albada and MC slopes, the HLLC and LLF
// fluxes, and the FP64 division, reciprocal and conversion helpers. The exact
// two-material Riemann solver of the FIVER flux is in m2c_riemann.cuh.
//
// Real type R is double on the FP64 path and float for the reconstruction and
// HLLC of the mixed-precision path; the Riemann solver is FP64 on both paths.
#pragma once
#include <cmath>
#include <cstdint>

#include "m2c.h"

namespace m2c {

// ---------------------------------------------------------------------------
// Equation of state parameters in device memory. SG: p = (g - 1) rho e - g pc
// (NASG of Sec. 3.3 with b = e_c = 0). MG: App. B.3 with the compression,
// tension and cutoff branches of the reference curves. NASG (Sec. 3.3, Eq.
// NASG_EOS): p = (g - 1) rho (e - e_c)/(1 - rho b) - g pc. JWL (App. B.2, Eq.
// JWL_EOS with the sign of its first exponential read as that of the second):
// p = w rho e + sum_i A_i (1 - w rho/(R_i rho0)) exp(-R_i rho0/rho).
// The NASG and JWL branches are compiled only where EXT is set (the general
// bulk kernel, the interface and Riemann kernels).
// ---------------------------------------------------------------------------
template <typename R>
struct EosP {
  int type;  // m2c_eos_type
  int pad;
  R g, pc, gm1, gpc, inv_gm1;                // SG and NASG
  R rho0, c0, s, G0, e0, eta_min;            // MG
  R K0, rg, inv_rg, inv_2rho0, eta_max, pmin, rk4_span;  // MG derived
  R b, ec;                                   // NASG
  R om, A1, A2, R1r, R2r, c1, c2;            // JWL: w, A_i, R_i rho0, w/(R_i rho0)
};
using EosDev = EosP<double>;

// Parameters computed in FP64 and rounded once to R.
template <typename R>
__host__ inline EosP<R> make_eos(int type, const double* prm) {
  EosP<R> e{};
  e.type = type;
  if (type == M2C_EOS_SG) {
    e.g = (R)prm[0];
    e.pc = (R)prm[1];
    e.gm1 = (R)(prm[0] - 1.0);
    e.gpc = (R)(prm[0] * prm[1]);
    e.inv_gm1 = (R)(1.0 / (prm[0] - 1.0));
  } else if (type == M2C_EOS_NASG) {
    e.g = (R)prm[0];
    e.pc = (R)prm[1];
    e.gm1 = (R)(prm[0] - 1.0);
    e.gpc = (R)(prm[0] * prm[1]);
    e.inv_gm1 = (R)(1.0 / (prm[0] - 1.0));
    e.b = (R)prm[2];
    e.ec = (R)prm[3];
  } else if (type == M2C_EOS_JWL) {
    e.om = (R)prm[0];
    e.A1 = (R)prm[1];
    e.A2 = (R)prm[2];
    e.R1r = (R)(prm[3] * prm[5]);
    e.R2r = (R)(prm[4] * prm[5]);
    e.c1 = (R)(prm[0] / (prm[3] * prm[5]));
    e.c2 = (R)(prm[0] / (prm[4] * prm[5]));
    e.rho0 = (R)prm[5];
  } else {
    const double K0 = prm[0] * prm[1] * prm[1], rg = prm[0] * prm[3];
    e.rho0 = (R)prm[0];
    e.c0 = (R)prm[1];
    e.s = (R)prm[2];
    e.G0 = (R)prm[3];
    e.e0 = (R)prm[4];
    e.eta_min = (R)prm[5];
    e.K0 = (R)K0;
    e.rg = (R)rg;
    e.inv_rg = (R)(1.0 / rg);
    e.inv_2rho0 = (R)(0.5 / prm[0]);
    e.eta_max = (R)(1.0 / prm[2]);
    e.pmin = (R)(K0 * prm[5]);
    e.rk4_span = (R)(0.05 * K0);
  }
  return e;
}

__host__ inline EosDev make_eos_dev(int type, const double* prm) { return make_eos<double>(type, prm); }

// Division, reciprocal and square root of the working precision. FP64: the
// quotient and reciprocal of div_nr / rcp_nr below (a binary32 seed refined by
// Newton-Raphson steps; the quotient takes a residual correction and equals the
// IEEE quotient, the reciprocal is within an ulp), IEEE square root. FP32 half
// of the mixed path: the hardware approximations (a few ulp), far below the
// FP32 rounding already accepted there.
__device__ __forceinline__ double rcp_nr(double b);
__device__ __forceinline__ double div_nr(double a, double b);
__device__ __forceinline__ bool nr_range(double b);
__device__ __forceinline__ double rcp_nr_in_range(double b);
template <typename R>
__device__ __forceinline__ R rdiv(R a, R b) {
  if constexpr (sizeof(R) == 8) return div_nr(a, b);
  else return __fdividef(a, b);
}
template <typename R>
__device__ __forceinline__ R rrcp(R x) {
  if constexpr (sizeof(R) == 8) return rcp_nr(x);
  else return __fdividef(1.0f, x);
}
template <typename R>
__device__ __forceinline__ R rsqrt_pos(R x) {  // sqrt of x > 0
  if constexpr (sizeof(R) == 8) return sqrt(x);
  else return x * rsqrtf(x);
}

// Exact IEEE-754 binary64 <-> binary32 conversions written with 32-bit
// integer operations (from the bit layout of the two formats), for the
// mixed-precision loads and updates: GB300 runs its conversion instructions on
// the narrow FP64 pipe (measured: about 600 G conversions/s per GPU, against
// 1.6 T for d2f below). d2f rounds to nearest, ties to even, including
// results in the binary32 subnormal range and overflow to infinity; a NaN
// stays a NaN. Host-callable so that they can be checked against the host's
// conversions.
__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double double_of(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  __builtin_memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned bits_of(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned b;
  __builtin_memcpy(&b, &x, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  __builtin_memcpy(&x, &b, 4);
  return x;
#endif
}

// The two 32-bit words of a binary64 value and back (register moves on the
// device). The helpers below work on these words: on GB300 a 64-bit integer
// operation costs several 32-bit ones, and the FP64 pipe is narrow.
__host__ __device__ __forceinline__ unsigned hi_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(x);
#else
  return (unsigned)(bits_of(x) >> 32);
#endif
}
__host__ __device__ __forceinline__ unsigned lo_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(x);
#else
  return (unsigned)bits_of(x);
#endif
}
__host__ __device__ __forceinline__ double double_of_words(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  return double_of(((unsigned long long)hi << 32) | lo);
#endif
}

// x < 0 and x > 0 for a binary64 x, decided on its bits (false for zeros of
// either sign and for NaNs; the infinities count), so that sign tests of FP64
// data stay off the FP64 pipe.
__host__ __device__ __forceinline__ bool lt0(double x) {
  const unsigned hi = hi_of(x), lo = lo_of(x);
  return (hi - 0x80000001u < 0x7fefffffu) || (hi == 0x80000000u && lo != 0u) || (hi == 0xfff00000u && lo == 0u);
}
__host__ __device__ __forceinline__ bool gt0(double x) {
  const unsigned hi = hi_of(x), lo = lo_of(x);
  return (hi - 1u < 0x7fefffffu) || (hi == 0u && lo != 0u) || (hi == 0x7ff00000u && lo == 0u);
}

// The cases outside the normal binary32 range (subnormal results, overflow,
// zeros, infinities, NaNs), out of line so that the common path stays short.
inline __host__ __device__ __noinline__ float d2f_rare(double x) {
  const unsigned long long b = bits_of(x);
  const unsigned long long a = b & 0x7fffffffffffffffull;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  unsigned r;
  if (a < 0x3810000000000000ull) {
    // |x| < 2^-126: result in units of 2^-149, M 2^(e-1075) = M 2^-(926-e) units
    const int e = (int)(a >> 52);
    if (e < 873) {
      r = 0u;  // below 2^-150 (exactly 2^-150 is handled below: a tie to even 0)
    } else {
      const unsigned long long M = (a & 0x000fffffffffffffull) | 0x0010000000000000ull;
      const int sh = 926 - e;  // 30 .. 53
      const unsigned long long q = M >> sh, rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
      r = (unsigned)(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
    }
  } else if (a <= 0x7ff0000000000000ull) {
    r = 0x7f800000u;  // |x| >= 2^128 and infinity
  } else {
    r = 0x7fc00000u | (unsigned)((a >> 29) & 0x003fffffull);  // quiet NaN
  }
  return float_of(r | sign);
}

__host__ __device__ __forceinline__ float d2f(double x) {
  const unsigned hi = hi_of(x), lo = lo_of(x), ah = hi & 0x7fffffffu;
  if (ah - 0x38100000u < 0x47f00000u - 0x38100000u) {
    // 2^-126 <= |x| < 2^128: rebias the exponent (1023 -> 127) and round the
    // 52-bit mantissa to 23 bits, ties to even, on the two words; a carry out
    // of the mantissa increments the exponent (at the top, to infinity)
    const unsigned r0 = ((ah - 0x38000000u) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    const unsigned r = r0 + ((rem > 0x10000000u || (rem == 0x10000000u && (r0 & 1u))) ? 1u : 0u);
    return float_of(r | (hi & 0x80000000u));
  }
  // zeros are common (momenta and residuals of a fluid at rest): kept on the inline path
  if ((ah | lo) == 0u) return float_of(hi);
  return d2f_rare(x);
}

inline __host__ __device__ __noinline__ double f2d_rare(float x) {
  const unsigned f = bits_of(x);
  const unsigned a = f & 0x7fffffffu;
  const unsigned long long sign = (unsigned long long)(f & 0x80000000u) << 32;
  unsigned long long r;
  if (a == 0u) {
    r = 0ull;
  } else if (a < 0x00800000u) {
    // subnormal a 2^-149: normalise the leading bit to position 23
#ifdef __CUDA_ARCH__
    const int s = __clz(a) - 8;
#else
    const int s = __builtin_clz(a) - 8;
#endif
    r = ((unsigned long long)(897 - s) << 52) | ((unsigned long long)((a << s) & 0x007fffffu) << 29);
  } else if (a == 0x7f800000u) {
    r = 0x7ff0000000000000ull;
  } else {
    r = 0x7ff8000000000000ull | ((unsigned long long)(a & 0x003fffffu) << 29);
  }
  return double_of(r | sign);
}

__host__ __device__ __forceinline__ double f2d(float x) {
  const unsigned f = bits_of(x), a = f & 0x7fffffffu;
  if (a - 0x00800000u < 0x7f800000u - 0x00800000u)  // normal: rebias 127 -> 1023
    return double_of_words(((a >> 3) + (896u << 20)) | (f & 0x80000000u), a << 29);
  if (a == 0u) return double_of_words(f, 0u);  // signed zero, inline
  return f2d_rare(x);
}

// A group of binary64 -> binary32 conversions (the plane loads of the mixed
// bulk kernel). On the device: the hardware conversion, round to nearest even,
// one instruction each on the FP64 pipe, which has room there once the update
// arithmetic is mostly FP32 (measured faster than the integer path for these
// loads, slower for the other conversions of the kernel). On the host: the
// common path of d2f (normal binary32 range and zeros) with one branch, to the
// exact d2f of every member, when a member falls outside it. Both give the
// IEEE result.
__host__ __device__ __forceinline__ float d2f_common(double x, bool& rare) {
  const unsigned hi = hi_of(x), lo = lo_of(x), ah = hi & 0x7fffffffu;
  const unsigned r0 = ((ah - 0x38000000u) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  const unsigned r = r0 + ((rem > 0x10000000u || (rem == 0x10000000u && (r0 & 1u))) ? 1u : 0u);
  const bool zero = (ah | lo) == 0u;
  rare = rare || !(ah - 0x38100000u < 0x47f00000u - 0x38100000u || zero);
  return float_of((zero ? 0u : r) | (hi & 0x80000000u));
}

template <int K>
__host__ __device__ __forceinline__ void d2f_group(const double (&x)[K], float (&y)[K]) {
#ifdef __CUDA_ARCH__
#pragma unroll
  for (int i = 0; i < K; ++i) y[i] = __double2float_rn(x[i]);
#else
  bool rare = false;
#pragma unroll
  for (int i = 0; i < K; ++i) y[i] = d2f_common(x[i], rare);
  if (rare) {
#pragma unroll
    for (int i = 0; i < K; ++i) y[i] = d2f(x[i]);
  }
#endif
}

// FP64 reciprocal and quotient for the bulk kernels: a binary32 seed of 1/b
// (b's leading 23 mantissa bits, then the hardware's approximate binary32
// reciprocal; relative error below 2^-21 together), refined by two
// Newton-Raphson steps x <- x + x (1 - b x), each of which squares the
// relative error, to 1/b within an ulp; the quotient a x then takes one
// residual correction q <- q + (a - b q) x (Markstein, IBM J. Res. Dev. 34,
// 1990). The seed stays on the integer and special-function pipes. For |b|
// outside [2^-125, 2^125) (zeros, infinities, NaNs included) the IEEE
// operations. Both are checked against IEEE 1/b and a/b on the device.
__device__ __forceinline__ bool nr_range(double b) {
  return (hi_of(b) & 0x7fffffffu) - 0x38200000u < 0x47c00000u - 0x38200000u;
}
__device__ __forceinline__ double rcp_nr_in_range(double b) {
  const unsigned hi = hi_of(b), ah = hi & 0x7fffffffu;
  const float f = float_of((((ah - 0x38000000u) << 3) | (lo_of(b) >> 29)) | (hi & 0x80000000u));
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));
  const unsigned rb = bits_of(r), ra = rb & 0x7fffffffu;
  double x = double_of_words(((ra >> 3) + (896u << 20)) | (rb & 0x80000000u), ra << 29);
  x = fma(x, fma(-b, x, 1.0), x);
  x = fma(x, fma(-b, x, 1.0), x);
  return x;
}
__device__ __forceinline__ double rcp_nr(double b) {
  if (nr_range(b)) return rcp_nr_in_range(b);
  return 1.0 / b;
}
// FP64 reciprocal square root 1/sqrt(x), x > 0, for the Mie-Grueneisen
// isentrope integrand: a binary32 seed (x's leading 23 mantissa bits, then the
// hardware's approximate binary32 reciprocal square root, relative error below
// 2^-21), refined by two Newton-Raphson steps y <- y + y (1 - x y^2)/2 in FP64
// (each squares the relative error up to a factor 3/2), within an ulp or two of
// 1/sqrt(x); x outside [2^-125, 2^125) takes 1/sqrt(x) with the IEEE operations.
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!nr_range(x)) return 1.0 / sqrt(x);
  const unsigned hi = hi_of(x);
  const float f = float_of(((hi - 0x38000000u) << 3) | (lo_of(x) >> 29));
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));
  const unsigned rb = bits_of(r);
  double y = double_of_words((rb >> 3) + (896u << 20), rb << 29);
  y = fma(0.5 * y, fma(-x * y, y, 1.0), y);
  y = fma(0.5 * y, fma(-x * y, y, 1.0), y);
  return y;
}

// The corrected quotient is the IEEE one when it is a normal number and its
// residual a - b q does not underflow: with |b| in the seed range that holds
// for |a| in [2^-897, 2^898). A zero a gives the signed zero a (1/b); any other
// a outside that range (a quotient that could overflow or underflow, an
// infinity, a NaN) takes the IEEE operation.
__device__ __forceinline__ double div_nr(double a, double b) {
  if (nr_range(b)) {
    const double x = rcp_nr_in_range(b), q = a * x;
    const unsigned ha = hi_of(a), ea = (ha >> 20) & 0x7ffu;
    if (ea - 126u < 1795u) return fma(fma(-b, q, a), x, q);
    if (((ha & 0x7fffffffu) | lo_of(a)) == 0u) return q;
  }
  return a / b;
}

template <typename R>
__device__ __forceinline__ R to_r(double x) {
  if constexpr (sizeof(R) == 8) return x;
  else return d2f(x);
}
template <typename R>
__device__ __forceinline__ double to_d(R x) {
  if constexpr (sizeof(R) == 8) return x;
  else return f2d(x);
}

// x > 0; FP64 values are tested on their bits (false for NaN either way), which
// keeps the comparison off the narrow FP64 pipe.
template <typename R>
__device__ __forceinline__ bool pos(R x) {
  if constexpr (sizeof(R) == 8) return gt0(x);
  else return x > (R)0;
}

// Reference curves p_R, p_R', e_R, e_R' at strain eta (App. B.3); "p_H" in the
// compression e_R is read as p_R.
template <typename R>
__device__ __forceinline__ void mg_ref(const EosP<R>& q, R eta, R& pR, R& dpR, R& eR, R& deR) {
  const R K0 = q.K0, rho0 = q.rho0, e0 = q.e0, h2 = q.inv_2rho0;
  if (pos(eta)) {
    R d = (R)1 - q.s * eta;
    R id = rrcp<R>(d);
    R id2 = id * id;
    pR = K0 * eta * id2;
    dpR = K0 * ((R)1 + q.s * eta) * id2 * id;
    eR = pR * eta * h2 + e0;
    deR = (dpR * eta + pR) * h2;
  } else if (eta >= q.eta_min) {
    pR = K0 * eta;
    dpR = K0;
    eR = K0 * eta * eta * h2 + e0;
    deR = K0 * eta * ((R)2 * h2);
  } else {
    R em = q.eta_min, pm = q.pmin;
    pR = pm;
    dpR = (R)0;
    eR = K0 * em * em * h2 + e0 + pm / rho0 * (eta - em);
    deR = pm / rho0;
  }
}

// JWL: f(rho) = sum_i A_i (1 - w rho/(R_i rho0)) exp(-R_i rho0/rho) and f'(rho).
template <typename R>
__device__ __forceinline__ void jwl_f(const EosP<R>& q, R rho, R inv_rho, R& f, R& df) {
  const R x1 = q.R1r * inv_rho, x2 = q.R2r * inv_rho;
  const R e1 = exp(-x1), e2 = exp(-x2);
  const R a1 = (R)1 - q.c1 * rho, a2 = (R)1 - q.c2 * rho;
  f = q.A1 * a1 * e1 + q.A2 * a2 * e2;
  df = q.A1 * e1 * (-q.c1 + a1 * x1 * inv_rho) + q.A2 * e2 * (-q.c2 + a2 * x2 * inv_rho);
}

// Material type test: T >= 0 is a type fixed at compile time (the bulk kernel's
// instantiations for one pair of SG / MG materials), T = -1 reads it from q.
template <int T, typename R>
__device__ __forceinline__ bool eos_is(const EosP<R>& q, int type) {
  if constexpr (T >= 0) return T == type;
  else return q.type == type;
}

// p(rho, e) given 1/rho; false if the state is outside the EOS domain.
template <typename R, bool EXT = false, int T = -1>
__device__ __forceinline__ bool eos_p(const EosP<R>& q, R rho, R inv_rho, R e, R& p) {
  if (eos_is<T>(q, M2C_EOS_SG)) {
    p = q.gm1 * rho * e - q.gpc;
    return true;
  }
  if constexpr (EXT) {
    if (q.type == M2C_EOS_NASG) {
      const R d = (R)1 - rho * q.b;
      if (!(d > (R)0)) return false;
      p = rdiv<R>(q.gm1 * rho * (e - q.ec), d) - q.gpc;
      return true;
    }
    if (q.type == M2C_EOS_JWL) {
      R f, df;
      jwl_f<R>(q, rho, inv_rho, f, df);
      p = q.om * rho * e + f;
      return true;
    }
  }
  R eta = (R)1 - q.rho0 * inv_rho;
  if (!(eta < q.eta_max)) return false;
  R pR, dpR, eR, deR;
  mg_ref(q, eta, pR, dpR, eR, deR);
  p = pR + q.rg * (e - eR);
  return true;
}

// e(rho, p) and c^2(rho, p) together (App. B.3 and App. C.2: c^2 = dp/drho|_e + p/rho^2 dp/de|_rho).
// False if rho <= 0, c^2 <= 0 or the state is outside the EOS domain.
template <typename R, bool EXT = false, int T = -1>
__device__ __forceinline__ bool eos_e_c2(const EosP<R>& q, R rho, R inv_rho, R p, R& e, R& c2) {
  if (!pos(rho)) return false;
  if (eos_is<T>(q, M2C_EOS_SG)) {
    R pb = p + q.pc;
    e = (p + q.gpc) * q.inv_gm1 * inv_rho;
    c2 = q.g * pb * inv_rho;
  } else if (EXT && q.type == M2C_EOS_NASG) {
    // e = e_c + (p + g pc)(1 - rho b)/((g - 1) rho), c^2 = g (p + pc)/(rho (1 - rho b))
    const R d = (R)1 - rho * q.b;
    if (!(d > (R)0)) return false;
    e = q.ec + (p + q.gpc) * d * q.inv_gm1 * inv_rho;
    c2 = rdiv<R>(q.g * (p + q.pc) * inv_rho, d);
  } else if (EXT && q.type == M2C_EOS_JWL) {
    // e = (p - f)/(w rho), c^2 = ((1 + w) p - f)/rho + f'
    R f, df;
    jwl_f<R>(q, rho, inv_rho, f, df);
    e = rdiv<R>((p - f) * inv_rho, q.om);
    c2 = ((R)1 + q.om) * p * inv_rho - f * inv_rho + df;
  } else {
    R eta = (R)1 - q.rho0 * inv_rho;
    if (!(eta < q.eta_max)) return false;
    R pR, dpR, eR, deR;
    mg_ref(q, eta, pR, dpR, eR, deR);
    e = eR + (p - pR) * q.inv_rg;
    R ir2 = inv_rho * inv_rho;
    c2 = ((dpR - q.rg * deR) * q.rho0 + p * q.rg) * ir2;
  }
  if constexpr (sizeof(R) == 8) return gt0(c2) && hi_of(c2) < 0x7ff00000u;
  else return c2 > (R)0 && c2 < (R)INFINITY;
}

// ---------------------------------------------------------------------------
// Modified van Albada slope (App. D, uniform grid A = B = 1, k = 2):
// sigma = a b (a + b)/(a^2 + b^2) when a b > 0, else 0.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R va_slope(R a, R b) {
  R ab = a * b;
  if constexpr (sizeof(R) == 8) {
    // FP64: the sign test on the bits and the quotient as the product with the
    // Newton-Raphson reciprocal (within an ulp or two of the IEEE quotient, which
    // is taken where the denominator is outside the reciprocal's range)
    if (!gt0(ab)) return 0.0;
    const double num = ab * (a + b), den = a * a + b * b;
    return nr_range(den) ? num * rcp_nr_in_range(den) : num / den;
  } else {
    if (!(ab > (R)0)) return (R)0;
    return rdiv<R>(ab * (a + b), a * a + b * b);
  }
}

// Monotonized central slope (App. D, Eq. theta) on the uniform grid, written
// without the division by b: sigma = phi(a/b) b with
// phi = max(0, min(alpha theta, (theta + 1)/2, alpha)); the inequalities turn
// for b < 0, and b = 0 gives 0.
template <typename R>
__device__ __forceinline__ R mc_slope(R a, R b, R alpha) {
  if (b > (R)0) return fmax((R)0, fmin(fmin(alpha * a, (R)0.5 * (a + b)), alpha * b));
  if (b < (R)0) return fmin((R)0, fmax(fmax(alpha * a, (R)0.5 * (a + b)), alpha * b));
  return (R)0;
}

// A reconstructed face state with its sound speed and total energy per mass.
template <typename R>
struct FaceState {
  R rho, u, v, w, p, c, E;
};

template <int D, typename R>
__device__ __forceinline__ R comp(const FaceState<R>& q) {
  return D == 0 ? q.u : (D == 1 ? q.v : q.w);
}

// Physical flux F(W).e_d (Sec. 3.2, Eq. NSEquation_terms) of a face state.
template <int D, typename R>
__device__ __forceinline__ void phys_flux(const FaceState<R>& q, R F[5]) {
  R un = comp<D>(q);
  R m = q.rho * un;
  F[0] = m;
  F[1] = m * q.u;
  F[2] = m * q.v;
  F[3] = m * q.w;
  F[1 + D] += q.p;
  F[4] = (q.rho * q.E + q.p) * un;
}

// HLLC flux (App. C.4): Davis wave speeds S_L = min(u_L - c_L, u_R - c_R),
// S_R = max(u_L + c_L, u_R + c_R), the contact speed S* as printed, and
// F* = F_K + S_K (W*_K - W_K) with W*_K = rho_K (S_K - u_K)/(S_K - S*) [1, V*, E*_K],
// V* normal = S*, tangential = side K's, E*_K = E_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K))).
template <int D, typename R>
__device__ __forceinline__ void hllc(const FaceState<R>& L, const FaceState<R>& Rt, R F[5]) {
  const R uL = comp<D>(L), uR = comp<D>(Rt);
  const R SL = fmin(uL - L.c, uR - Rt.c);
  const R SR = fmax(uL + L.c, uR + Rt.c);
  const R aL = L.rho * (SL - uL), aR = Rt.rho * (SR - uR);
  const R Ss = rdiv<R>(Rt.p - L.p + uL * aL - uR * aR, aL - aR);
  if ((R)0 <= SL) {
    phys_flux<D>(L, F);
    return;
  }
  bool left;
  if ((R)0 <= Ss) left = true;
  else if ((R)0 <= SR) left = false;
  else {
    phys_flux<D>(Rt, F);
    return;
  }
  const FaceState<R>& K = left ? L : Rt;
  const R SK = left ? SL : SR;
  const R uK = left ? uL : uR;
  const R aK = left ? aL : aR;
  phys_flux<D>(K, F);
  const R fac = rdiv<R>(aK, SK - Ss);
  const R Es = K.E + (Ss - uK) * (Ss + rdiv<R>(K.p, aK));
  R ws[5] = {fac, fac * K.u, fac * K.v, fac * K.w, fac * Es};
  ws[1 + D] = fac * Ss;
  const R wk[5] = {K.rho, K.rho * K.u, K.rho * K.v, K.rho * K.w, K.rho * K.E};
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = F[v] + SK * (ws[v] - wk[v]);
}

// Local Lax-Friedrichs flux (App. C.1, Eq. Lax-Friedrichs):
// F = (F(W_L) + F(W_R))/2 - lambda (W_R - W_L)/2 with
// lambda = max(|u_L| + c_L, |u_R| + c_R), u the normal velocities.
template <int D, typename R>
__device__ __forceinline__ void llf(const FaceState<R>& L, const FaceState<R>& Rt, R F[5]) {
  const R lam = fmax(fabs(comp<D>(L)) + L.c, fabs(comp<D>(Rt)) + Rt.c);
  R FL[5], FR[5];
  phys_flux<D>(L, FL);
  phys_flux<D>(Rt, FR);
  const R wL[5] = {L.rho, L.rho * L.u, L.rho * L.v, L.rho * L.w, L.rho * L.E};
  const R wR[5] = {Rt.rho, Rt.rho * Rt.u, Rt.rho * Rt.v, Rt.rho * Rt.w, Rt.rho * Rt.E};
  const R hl = (R)0.5 * lam;
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = (R)0.5 * (FL[v] + FR[v]) - hl * (wR[v] - wL[v]);
}

// The grid's numerical flux: HLLC, or (general kernels, flux = M2C_FLUX_LLF) LLF.
template <int D, typename R, bool GEN>
__device__ __forceinline__ void num_flux(const FaceState<R>& L, const FaceState<R>& Rt, R F[5], int flux) {
  if constexpr (GEN) {
    if (flux == M2C_FLUX_LLF) {
      llf<D, R>(L, Rt, F);
      return;
    }
  }
  hllc<D, R>(L, Rt, F);
}

}  // namespace m2c
