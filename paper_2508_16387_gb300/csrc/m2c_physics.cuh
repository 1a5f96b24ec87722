// Device-side physics of the M2C finite-volume step (arXiv 2508.16387):
// equations of state, the modified van Albada slope, the HLLC flux and the
// exact two-material Riemann solver of the FIVER flux.
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

// A group of d2f conversions taken on the common path (normal binary32 range
// and zeros) with one branch, to the exact d2f of every member, when a member
// falls outside it: the same results as d2f, and the group stays one basic
// block in the common case.
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
  bool rare = false;
#pragma unroll
  for (int i = 0; i < K; ++i) y[i] = d2f_common(x[i], rare);
  if (rare) {
#pragma unroll
    for (int i = 0; i < K; ++i) y[i] = d2f(x[i]);
  }
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

// ---------------------------------------------------------------------------
// Exact two-material Riemann problem (Sec. 4.2, Eq. 1DRiemannProblem with the
// interface conditions of Sec. 3.5.1), FP64. Newton on p* from the PVRS guess,
// stop at the first step with |dp| <= 1e-12 |p|; 50 steps then bisection.
// SG wave curves in closed form; MG shock from the Hugoniot root, MG
// rarefaction by RK4 on equal pressure substeps whose number is fixed once
// per problem (fix_substeps) from a bound of the wave's pressure span.
// ---------------------------------------------------------------------------
constexpr double kNewtonTol = 1e-12;
constexpr int kNewtonCap = 50;
constexpr int kBisectCap = 200;
constexpr double kHugTol = 1e-14;
constexpr int kHugCap = 100;
constexpr int kRk4Steps = 64;

struct Side {
  double rho, u, p, c, e;
  int nrk;  // RK4 substeps of this side's MG rarefaction curve in one problem; 0: per evaluation
  // MG: spacing of the problem's fixed RK4 nodes p_K - i dnode (0: none), and the
  // isentrope state (rho, f) after the first mbase full substeps, kept between the
  // evaluations of one problem (nearby pressures share their nodes)
  int mbase;
  double dnode, dspan, rbase, fbase;  // dspan = nrk dnode, the span bound the nodes cover
};

__device__ inline bool make_side(const EosDev& q, double rho, double u, double p, Side& K) {
  if (!(rho > 0.0)) return false;
  double e, c2;
  if (!eos_e_c2<double, true>(q, rho, 1.0 / rho, p, e, c2)) return false;
  K.rho = rho;
  K.u = u;
  K.p = p;
  K.c = sqrt(c2);
  K.e = e;
  K.nrk = 0;
  K.mbase = 0;
  K.dnode = 0.0;
  K.dspan = 0.0;
  K.rbase = rho;
  K.fbase = 0.0;
  return true;
}

// Lowest admissible pressure of a side: p + p_c > 0 (SG, NASG), p > 0 (JWL,
// whose rarefaction is integrated in ln p), the MG tensile cutoff if any.
__device__ inline double eos_plow(const EosDev& q) {
  if (q.type == M2C_EOS_SG || q.type == M2C_EOS_NASG) return -q.pc;
  if (q.type == M2C_EOS_JWL) return 0.0;
  return isfinite(q.eta_min) ? q.pmin : -INFINITY;
}

// Equal RK4 substeps over a pressure span dp of an MG isentrope: 64 for a span
// of at least 5% of K0 = rho0 c0^2, proportionally fewer (at least one) below.
__device__ inline int mg_substeps(const EosDev& q, double dp) {
  double nsd = ceil(__ddiv_rn(kRk4Steps * fabs(dp), q.rk4_span));
  nsd = nsd >= 1.0 ? (nsd > kRk4Steps ? (double)kRk4Steps : nsd) : 1.0;
  return (int)nsd;
}

// JWL rarefactions are integrated in ln p (detonation products expand over
// decades): 256 substeps per unit of ln(p_K/p_lo), at least 8, with p_lo kept
// at or above 1e-6 p_K.
__device__ inline int jwl_substeps(double pK, double p_lo) {
  const double lo = fmax(p_lo, 1e-6 * pK);
  const double nd = ceil(256.0 * log(pK / lo));
  return nd < 8.0 ? 8 : (int)nd;
}

// The substep count of each MG side's rarefaction curve, fixed once per
// problem before the iteration so that the curve is one smooth function of p:
// the count for an upper bound of the pressure drop across the wave,
// p_K - max(p_low, min(p_J, p_ac)), with the acoustic estimate
// p_ac = (Z_R p_L + Z_L p_R - Z_L Z_R (u_R - u_L)) / (Z_L + Z_R), Z = rho c
// (a shock on the other side J keeps p* above p_J; a rarefaction there too
// keeps p* above p_ac, since each rarefaction curve lies below its acoustic
// tangent). Written without contracted multiply-adds.
__device__ inline void fix_substeps(const EosDev& qL, Side& L, const EosDev& qR, Side& Rs, double plow) {
  const double ZL = __dmul_rn(L.rho, L.c), ZR = __dmul_rn(Rs.rho, Rs.c);
  const double num = __dsub_rn(__dadd_rn(__dmul_rn(ZR, L.p), __dmul_rn(ZL, Rs.p)),
                               __dmul_rn(__dmul_rn(ZL, ZR), __dsub_rn(Rs.u, L.u)));
  const double pac = __ddiv_rn(num, __dadd_rn(ZL, ZR));
  const double loL = fmax(plow, fmin(Rs.p, pac)), loR = fmax(plow, fmin(L.p, pac));
  // MG: the count for the span bound and the spacing of the fixed nodes (span / count)
  auto mg_nodes = [](const EosDev& q, Side& K, double lo) {
    const double span = fmax(__dsub_rn(K.p, lo), 0.0);
    K.nrk = mg_substeps(q, span);
    K.dnode = (span > 0.0 && isfinite(span)) ? __ddiv_rn(span, (double)K.nrk) : 0.0;
    K.dspan = __dmul_rn((double)K.nrk, K.dnode);
  };
  if (qL.type == M2C_EOS_MG) mg_nodes(qL, L, loL);
  if (qR.type == M2C_EOS_MG) mg_nodes(qR, Rs, loR);
  if (qL.type == M2C_EOS_JWL) L.nrk = jwl_substeps(L.p, loL);
  if (qR.type == M2C_EOS_JWL) Rs.nrk = jwl_substeps(Rs.p, loR);
}

__device__ inline int wave_sg(const EosDev& q, const Side& K, double p, double& f, double& df, double& rs,
                              bool want_rho = true, double* drs = nullptr) {
  const double g = q.g, pb = p + q.pc, pbK = K.p + q.pc;
  if (!(pb >= 0.0) || !(pbK > 0.0)) return M2C_ENONPHYS;
  if (p > K.p) {
    double A = 2.0 / ((g + 1.0) * K.rho);
    double B = (g - 1.0) / (g + 1.0) * pbK;
    double sq = sqrt(A / (pb + B));
    f = (p - K.p) * sq;
    df = sq * (1.0 - 0.5 * (p - K.p) / (pb + B));
    double r = pb / pbK, gm = (g - 1.0) / (g + 1.0);
    rs = K.rho * (r + gm) / (gm * r + 1.0);
    if (drs) *drs = K.rho * (1.0 - gm * gm) / ((gm * r + 1.0) * (gm * r + 1.0) * pbK);
  } else {
    // one power serves f and f': r^{-(g+1)/(2g)} = r^{(g-1)/(2g)} / r; the density
    // behind the wave is only evaluated when asked for (after the iteration)
    const double r = pb / pbK;
    const double q = pow(r, (g - 1.0) / (2.0 * g));
    f = 2.0 * K.c / (g - 1.0) * (q - 1.0);
    df = q / (r * K.rho * K.c);
    rs = want_rho ? K.rho * pow(r, 1.0 / g) : 0.0;
    if (drs) *drs = rs / (g * pb);
  }
  return M2C_OK;
}

// de/drho at constant p for MG
__device__ inline bool mg_dedr(const EosDev& q, double rho, double& dedr) {
  double eta = 1.0 - div_nr(q.rho0, rho);
  if (!(eta < q.eta_max)) return false;
  double pR, dpR, eR, deR;
  mg_ref<double>(q, eta, pR, dpR, eR, deR);
  dedr = div_nr((deR - dpR * q.inv_rg) * q.rho0, rho * rho);
  return true;
}

// Density on the MG Hugoniot through K at pressure p (safeguarded Newton in a
// closed bracket, stopped at the first step below the tolerance) and d rho/dp
// along it.
__device__ inline int mg_hugoniot(const EosDev& q, const Side& K, double p, double& rho_out, double& drdp) {
  double lo = K.rho, hi = q.rho0 * q.s / (q.s - 1.0);
  if (!(hi > lo)) return M2C_ENONPHYS;
  double rho = K.rho + div_nr(p - K.p, K.c * K.c);
  if (!(rho > lo && rho < hi)) rho = 0.5 * (lo + hi);
  bool done = false;
  for (int it = 0; it < kHugCap; ++it) {
    double eta = 1.0 - div_nr(q.rho0, rho);
    if (!(eta < q.eta_max)) return M2C_ENONPHYS;
    double pR, dpR, eR, deR;
    mg_ref<double>(q, eta, pR, dpR, eR, deR);
    double e = eR + (p - pR) * q.inv_rg;
    double dedr = div_nr((deR - dpR * q.inv_rg) * q.rho0, rho * rho);
    double H = e - K.e - 0.5 * (p + K.p) * (div_nr(1.0, K.rho) - div_nr(1.0, rho));
    double dH = dedr - div_nr(0.5 * (p + K.p), rho * rho);
    if (H > 0.0) lo = rho; else hi = rho;
    double rn = rho - div_nr(H, dH);
    if (!(rn >= lo && rn <= hi)) rn = 0.5 * (lo + hi);
    bool conv = fabs(rn - rho) <= kHugTol * rn;
    rho = rn;
    if (conv) { done = true; break; }
  }
  if (!done) return M2C_ENOCONV;
  double dedr;
  if (!mg_dedr(q, rho, dedr)) return M2C_ENONPHYS;
  double Hp = q.inv_rg - 0.5 * (div_nr(1.0, K.rho) - div_nr(1.0, rho));
  double Hr = dedr - div_nr(0.5 * (p + K.p), rho * rho);
  rho_out = rho;
  drdp = -div_nr(Hp, Hr);
  return M2C_OK;
}

// d rho/dp = 1/c^2 and df/dp = 1/(rho c) of the isentrope from one reciprocal
// square root of c^2 and the reciprocal of rho (each within an ulp or two of the
// correctly rounded value).
__device__ inline int mg_rhs(const EosDev& q, double p, double rho, double& drho, double& dfv) {
  double e, c2;
  const double ir = rcp_nr(rho);
  if (!eos_e_c2<double>(q, rho, ir, p, e, c2)) return M2C_ENONPHYS;
  const double y = rsqrt_nr(c2);
  drho = y * y;
  dfv = y * ir;
  return M2C_OK;
}

// One classical RK4 substep of the MG isentrope (rho, f) from pressure pi by hs.
__device__ inline int mg_rk4_substep(const EosDev& q, double pi, double hs, double& rho, double& fv) {
  double k1r, k1f, k2r, k2f, k3r, k3f, k4r, k4f;
  int st = mg_rhs(q, pi, rho, k1r, k1f);
  if (!st) st = mg_rhs(q, pi + 0.5 * hs, rho + 0.5 * hs * k1r, k2r, k2f);
  if (!st) st = mg_rhs(q, pi + 0.5 * hs, rho + 0.5 * hs * k2r, k3r, k3f);
  if (!st) st = mg_rhs(q, pi + hs, rho + hs * k3r, k4r, k4f);
  if (st) return st;
  rho = rho + hs / 6.0 * (k1r + 2.0 * k2r + 2.0 * k3r + k4r);
  fv = fv + hs / 6.0 * (k1f + 2.0 * k2f + 2.0 * k3f + k4f);
  return M2C_OK;
}

// MG wave curve. Rarefaction: the isentrope integrated by classical RK4 in p;
// inside a problem's span bound on the fixed nodes p_K - i dnode (full substeps
// down to the last node above p, resumed from the node reached by an earlier
// evaluation of the problem when it lies at or below, then one partial substep
// to p): the curve is continuous and smooth in p; beyond the bound, and for a
// wave evaluated alone, equal substeps over p_K - p. The node arithmetic is
// written without contracted multiply-adds, so that it takes the same nodes as
// the oracle.
__device__ inline int wave_mg(const EosDev& q, Side& K, double p, double& f, double& df, double& rs,
                              double* drs = nullptr) {
  if (p == K.p) {
    f = 0.0;
    df = 1.0 / (K.rho * K.c);
    rs = K.rho;
    if (drs) *drs = 1.0 / (K.c * K.c);
    return M2C_OK;
  }
  if (p > K.p) {
    double rho, drdp;
    int st = mg_hugoniot(q, K, p, rho, drdp);
    if (st) return st;
    double dv = div_nr(1.0, K.rho) - div_nr(1.0, rho);
    double fv = sqrt((p - K.p) * dv);
    f = fv;
    df = div_nr(dv + div_nr((p - K.p) * drdp, rho * rho), 2.0 * fv);
    rs = rho;
    if (drs) *drs = drdp;
    return M2C_OK;
  }
  double rho = K.rho, fv = 0.0;
  const double dp = __dsub_rn(K.p, p);
  // (one node interval: the partial substep from p_K is the single equal substep
  // over p_K - p, the same arithmetic, so that case takes the short path)
  if (K.nrk > 1 && K.dnode > 0.0 && dp < K.dspan) {
    int m = (int)floor(div_nr(dp, K.dnode));  // div_nr: the IEEE quotient
    if (m > K.nrk - 1) m = K.nrk - 1;
    if (K.mbase > m) {  // an earlier evaluation went past this node: start over from p_K
      K.mbase = 0;
      K.rbase = K.rho;
      K.fbase = 0.0;
    }
    rho = K.rbase;
    fv = K.fbase;
    for (int i = K.mbase; i < m; ++i) {
      const int st = mg_rk4_substep(q, __dsub_rn(K.p, __dmul_rn((double)i, K.dnode)), -K.dnode, rho, fv);
      if (st) return st;
    }
    K.mbase = m;
    K.rbase = rho;
    K.fbase = fv;
    const double hp = __dsub_rn(dp, __dmul_rn((double)m, K.dnode));
    if (hp > 0.0) {
      const int st = mg_rk4_substep(q, __dsub_rn(K.p, __dmul_rn((double)m, K.dnode)), -hp, rho, fv);
      if (st) return st;
    }
  } else {
    // equal substeps: the problem's count (beyond its span bound), else chosen for this span
    const int ns = K.nrk > 0 ? K.nrk : mg_substeps(q, p - K.p);
    const double hs = (p - K.p) / ns;
    for (int i = 0; i < ns; ++i) {
      const int st = mg_rk4_substep(q, K.p + i * hs, hs, rho, fv);
      if (st) return st;
    }
  }
  double e, c2;
  if (!eos_e_c2<double>(q, rho, 1.0 / rho, p, e, c2)) return M2C_ENONPHYS;
  f = fv;
  df = 1.0 / (rho * sqrt(c2));
  rs = rho;
  if (drs) *drs = 1.0 / c2;
  return M2C_OK;
}

// NASG wave curves in P = p + p_c and the covolume-reduced specific volume
// w = 1/rho - b. Shock: the Hugoniot energy equation is linear in w,
// w = w_K (gm r + 1)/(r + gm), r = P/P_K, gm = (g - 1)/(g + 1), so
// f = (p - p_K) sqrt(A/(P + gm P_K)) with A = 2 w_K/(g + 1). Rarefaction: the
// isentrope P w^g = const gives rho c = sqrt(g P / w) and
// f = 2 c_K (1 - b rho_K)/(g - 1) (r^((g-1)/(2g)) - 1).
static __device__ __noinline__ int wave_nasg(const EosDev& q, const Side& K, double p, double& f, double& df,
                                             double& rs, double* drs) {
  const double g = q.g, b = q.b, P = p + q.pc, PK = K.p + q.pc, wK = 1.0 / K.rho - b;
  if (!(P >= 0.0) || !(PK > 0.0) || !(wK > 0.0)) return M2C_ENONPHYS;
  const double r = P / PK;
  if (p > K.p) {
    const double gm = (g - 1.0) / (g + 1.0), A = 2.0 * wK / (g + 1.0), D = P + gm * PK;
    const double sq = sqrt(A / D);
    f = (p - K.p) * sq;
    df = sq * (1.0 - 0.5 * (p - K.p) / D);
    const double w = wK * (gm * r + 1.0) / (r + gm);
    rs = 1.0 / (b + w);
    if (drs) *drs = rs * rs * wK * (1.0 - gm * gm) / ((r + gm) * (r + gm) * PK);
  } else {
    f = 2.0 * K.c * (1.0 - b * K.rho) / (g - 1.0) * (pow(r, (g - 1.0) / (2.0 * g)) - 1.0);
    const double w = wK * pow(r, -1.0 / g);
    df = sqrt(w / (g * P));
    rs = 1.0 / (b + w);
    if (drs) *drs = rs * rs * w / (g * P);
  }
  return M2C_OK;
}

// JWL Hugoniot through K at p > p_K: the root rho > rho_K of
// H(rho) = e(rho, p) - e_K - (p + p_K)(1/rho_K - 1/rho)/2, bracketed from
// [rho_K, rho_K (w + 2)/w] (doubling the upper end until H < 0), then Newton
// kept inside the bracket with the tolerance and stopping rule of the MG root;
// d rho/dp by implicit differentiation. de/drho|_p = -(f'(rho) + w e)/(w rho).
__device__ inline int jwl_hugoniot(const EosDev& q, const Side& K, double p, double& rho_out, double& drdp) {
  const double w = q.om;
  double lo = K.rho, hi = K.rho * (w + 2.0) / w;
  bool bracketed = false;
  for (int k = 0; k < 60 && !bracketed; ++k) {
    double f, df;
    jwl_f<double>(q, hi, 1.0 / hi, f, df);
    const double e = (p - f) / (w * hi);
    if (e - K.e - 0.5 * (p + K.p) * (1.0 / K.rho - 1.0 / hi) < 0.0) bracketed = true;
    else { lo = hi; hi = 2.0 * hi; }
  }
  if (!bracketed) return M2C_ENOCONV;
  double rho = K.rho + (p - K.p) / (K.c * K.c);
  if (!(rho > lo && rho < hi)) rho = 0.5 * (lo + hi);
  bool done = false;
  for (int it = 0; it < kHugCap; ++it) {
    double f, df;
    jwl_f<double>(q, rho, 1.0 / rho, f, df);
    const double e = (p - f) / (w * rho);
    const double dedr = -(df + w * e) / (w * rho);
    const double H = e - K.e - 0.5 * (p + K.p) * (1.0 / K.rho - 1.0 / rho);
    const double dH = dedr - 0.5 * (p + K.p) / (rho * rho);
    if (H > 0.0) lo = rho; else hi = rho;
    double rn = rho - H / dH;
    if (!(rn >= lo && rn <= hi)) rn = 0.5 * (lo + hi);
    const bool conv = fabs(rn - rho) <= kHugTol * rn;
    rho = rn;
    if (conv) { done = true; break; }
  }
  if (!done) return M2C_ENOCONV;
  double f, df;
  jwl_f<double>(q, rho, 1.0 / rho, f, df);
  const double e = (p - f) / (w * rho);
  const double Hp = 1.0 / (w * rho) - 0.5 * (1.0 / K.rho - 1.0 / rho);
  const double Hr = -(df + w * e) / (w * rho) - 0.5 * (p + K.p) / (rho * rho);
  rho_out = rho;
  drdp = -Hp / Hr;
  return M2C_OK;
}

// JWL wave curve: shock f = sqrt((p - p_K)(1/rho_K - 1/rho_H(p))); rarefaction:
// the isentrope d rho/dp = 1/c^2, df/dp = 1/(rho c) integrated by classical RK4
// in s = ln p on equal substeps (fixed per problem, fix_substeps; else for
// this span); it needs p > 0.
static __device__ __noinline__ int wave_jwl(const EosDev& q, const Side& K, double p, double& f, double& df,
                                            double& rs, double* drs) {
  if (p == K.p) {
    f = 0.0;
    df = 1.0 / (K.rho * K.c);
    rs = K.rho;
    if (drs) *drs = 1.0 / (K.c * K.c);
    return M2C_OK;
  }
  if (p > K.p) {
    double rho, drdp;
    const int st = jwl_hugoniot(q, K, p, rho, drdp);
    if (st) return st;
    const double dv = 1.0 / K.rho - 1.0 / rho;
    const double fv = sqrt((p - K.p) * dv);
    f = fv;
    df = (dv + (p - K.p) * drdp / (rho * rho)) / (2.0 * fv);
    rs = rho;
    if (drs) *drs = drdp;
    return M2C_OK;
  }
  if (!(p > 0.0) || !(K.p > 0.0)) return M2C_ENONPHYS;
  const double span = log(p / K.p);
  int ns = K.nrk;
  if (ns <= 0) {
    const double nd = ceil(256.0 * fabs(span));
    ns = nd < 8.0 ? 8 : (int)nd;
  }
  const double hs = span / ns, s0 = log(K.p);
  double rho = K.rho, fv = 0.0;
  // d(rho, f)/ds at (s, rho): (p / c^2, p / (rho c)) with p = exp(s)
  auto rhs = [&](double si, double r, double& kr, double& kf) {
    const double pp = exp(si);
    double e, c2;
    if (!eos_e_c2<double, true>(q, r, 1.0 / r, pp, e, c2)) return false;
    kr = pp / c2;
    kf = pp / (r * sqrt(c2));
    return true;
  };
  for (int i = 0; i < ns; ++i) {
    const double si = s0 + i * hs;
    double k1r, k1f, k2r, k2f, k3r, k3f, k4r, k4f;
    if (!rhs(si, rho, k1r, k1f) || !rhs(si + 0.5 * hs, rho + 0.5 * hs * k1r, k2r, k2f) ||
        !rhs(si + 0.5 * hs, rho + 0.5 * hs * k2r, k3r, k3f) || !rhs(si + hs, rho + hs * k3r, k4r, k4f))
      return M2C_ENONPHYS;
    rho = rho + hs / 6.0 * (k1r + 2.0 * k2r + 2.0 * k3r + k4r);
    fv = fv + hs / 6.0 * (k1f + 2.0 * k2f + 2.0 * k3f + k4f);
  }
  double e, c2;
  if (!eos_e_c2<double, true>(q, rho, 1.0 / rho, p, e, c2)) return M2C_ENONPHYS;
  f = fv;
  df = 1.0 / (rho * sqrt(c2));
  rs = rho;
  if (drs) *drs = 1.0 / c2;
  return M2C_OK;
}

__device__ inline int wave(const EosDev& q, Side& K, double p, double& f, double& df, double& rs,
                           bool want_rho = true, double* drs = nullptr) {
  if (q.type == M2C_EOS_SG) return wave_sg(q, K, p, f, df, rs, want_rho, drs);
  if (q.type == M2C_EOS_MG) return wave_mg(q, K, p, f, df, rs, drs);
  if (q.type == M2C_EOS_NASG) return wave_nasg(q, K, p, f, df, rs, drs);
  return wave_jwl(q, K, p, f, df, rs, drs);
}

// Both wave curves at p: f and f' of each side, and on request (wv) the star
// densities behind the two waves and their slopes d rho*/dp as well.
struct WaveVals {
  double fL, dfL, rL, dL, fR, dfR, rR, dR;
};

static __device__ __noinline__ int riemann_F(const EosDev& qL, Side& L, const EosDev& qR, Side& Rs, double p,
                                double& F, double& dF, WaveVals* wv = nullptr) {
  double fL, dfL, rL, fR, dfR, rR, dL = 0.0, dR = 0.0;
  const bool want = wv != nullptr;
  int st = wave(qL, L, p, fL, dfL, rL, want, want ? &dL : nullptr);
  if (!st) st = wave(qR, Rs, p, fR, dfR, rR, want, want ? &dR : nullptr);
  if (st) return st;
  F = fL + fR + (Rs.u - L.u);
  dF = dfL + dfR;
  if (wv) *wv = WaveVals{fL, dfL, rL, dL, fR, dfR, rR, dR};
  return M2C_OK;
}

struct RiemannOut {
  double p, u, rhoL, rhoR;
};

// Solves the 1D problem between (rho, u, p) states; returns a status and the
// Newton/bisection iteration count. p_start: a start of the Newton iteration
// (the FIVER kernel passes the same face's star pressure of its previous
// solve); NaN, or a value not above the lowest admissible pressure, takes the
// PVRS estimate. The root and the stopping rule do not depend on the start.
static __device__ __noinline__ int riemann_solve(const EosDev& qL, double rl, double ul, double pl, const EosDev& qR, double rr,
                                    double ur, double pr, RiemannOut& out, int& iters,
                                    double p_start = NAN) {
  Side L, Rs;
  iters = 0;
  if (!make_side(qL, rl, ul, pl, L) || !make_side(qR, rr, ur, pr, Rs)) return M2C_ENONPHYS;
  const double plow = fmax(eos_plow(qL), eos_plow(qR));
  fix_substeps(qL, L, qR, Rs, plow);
  double F, dF;
  int st;
  // vacuum test (F(p_low) >= 0); both wave curves increase with p and vanish at
  // their side's pressure, so F(p_low) <= u_R - u_L and the test is only made
  // when u_R - u_L >= 0
  // no vacuum test with a JWL side (its rarefaction needs p > 0)
  if (isfinite(plow) && Rs.u - L.u >= 0.0 && qL.type != M2C_EOS_JWL && qR.type != M2C_EOS_JWL) {
    st = riemann_F(qL, L, qR, Rs, plow, F, dF);
    if (st) return st;
    if (F >= 0.0) return M2C_EVACUUM;
  }
  double p = 0.5 * (L.p + Rs.p) - 0.125 * (Rs.u - L.u) * (L.rho + Rs.rho) * (L.c + Rs.c);
  const bool warm = p_start > plow && p_start < INFINITY;
  if (warm) p = p_start;
  if (!(p > plow)) {
    double gap = fmin(L.p, Rs.p) - plow;
    if (!(gap > 0.0)) gap = fmax(L.p, Rs.p) - plow;
    p = plow + 1e-3 * gap;
  }
  int it;
  bool conv = false;
  // every evaluation also returns the star densities, so that the solution
  // follows from the last one to first order in its step (at most the
  // tolerance: the error is of the order of its square) instead of from one
  // more evaluation
  WaveVals wv{};
  double p_last = 0.0;
  for (it = 1; it <= kNewtonCap; ++it) {
    st = riemann_F(qL, L, qR, Rs, p, F, dF, &wv);
    if (st) return st;
    double pn = p - F / dF;
    if (!(pn > plow)) pn = 0.5 * (p + plow);
    bool small = fabs(pn - p) <= kNewtonTol * fabs(pn);
    p_last = p;
    p = pn;
    if (small) { conv = true; break; }
  }
  if (!conv) {
    double a = plow, b = fmax(L.p, Rs.p);
    if (!isfinite(a)) {
      a = fmin(L.p, Rs.p);
      for (int k = 0; k < kBisectCap; ++k) {
        st = riemann_F(qL, L, qR, Rs, a, F, dF);
        if (st) return st;
        if (F < 0.0) break;
        a = a - 2.0 * fabs(a) - 1.0;
      }
    }
    for (int k = 0; k < kBisectCap; ++k) {
      st = riemann_F(qL, L, qR, Rs, b, F, dF);
      if (st) return st;
      if (F > 0.0) break;
      b = 2.0 * b + fabs(b) + 1.0;
    }
    bool ok = false;
    for (int k = 0; k < kBisectCap; ++k) {
      double m = 0.5 * (a + b);
      st = riemann_F(qL, L, qR, Rs, m, F, dF);
      if (st) return st;
      if (F < 0.0) a = m; else b = m;
      ++it;
      if (b - a <= 1e-14 * fmax(fabs(a), fabs(b))) { ok = true; break; }
    }
    if (!ok) return M2C_ENOCONV;
    p = 0.5 * (a + b);
  }
  if (conv && isfinite(wv.dfL) && isfinite(wv.dfR) && isfinite(wv.dL) && isfinite(wv.dR)) {
    const double d = p - p_last;
    out.p = p;
    out.u = 0.5 * (L.u + Rs.u) + 0.5 * (wv.fR - wv.fL) + 0.5 * (wv.dfR - wv.dfL) * d;
    out.rhoL = wv.rL + wv.dL * d;
    out.rhoR = wv.rR + wv.dR * d;
    iters = it;
    return M2C_OK;
  }
  double fL, dfL, rL, fR, dfR, rR;
  st = wave(qL, L, p, fL, dfL, rL);
  if (!st) st = wave(qR, Rs, p, fR, dfR, rR);
  if (st) return st;
  out.p = p;
  out.u = 0.5 * (L.u + Rs.u) + 0.5 * (fR - fL);
  out.rhoL = rL;
  out.rhoR = rR;
  iters = it;
  return M2C_OK;
}

// ---------------------------------------------------------------------------
// Mixed-precision exact Riemann solve: Newton on p* first runs on FP32 wave
// curves (the same PVRS start and curves, with FP32 tolerances; weak waves of
// a stiff MG material, |p - p_K| <= 1e-5 rho_K c_K^2, take the acoustic
// curve, which is all an FP32 start can resolve there), then one FP64 Newton
// step from the FP32 root on the FP64 wave curves (two if the first moves p by
// more than 1e-9 |p|) gives p*; u* and the star densities follow from the last
// FP64 evaluation to first order in the step. An FP32 failure, a vacuum
// signal, a slope that is not finite, or a step larger than 1e-5 |p| leaves
// the problem to the FP64 iteration above.
// ---------------------------------------------------------------------------
struct SideF {
  float rho, u, p, c, e;
};

__device__ inline bool make_side_f(const EosP<float>& q, float rho, float u, float p, SideF& K) {
  if (!(rho > 0.0f)) return false;
  float e, c2;
  if (!eos_e_c2<float>(q, rho, 1.0f / rho, p, e, c2)) return false;
  K.rho = rho;
  K.u = u;
  K.p = p;
  K.c = sqrtf(c2);
  K.e = e;
  return true;
}

__device__ inline float eos_plow_f(const EosP<float>& q) {
  if (q.type == M2C_EOS_SG) return -q.pc;
  return isfinite(q.eta_min) ? q.pmin : -INFINITY;
}

__device__ inline bool wave_sg_f(const EosP<float>& q, const SideF& K, float p, float& f, float& df) {
  const float g = q.g, pb = p + q.pc, pbK = K.p + q.pc, dp = p - K.p;
  if (!(pb >= 0.0f) || !(pbK > 0.0f)) return false;
  if (p > K.p) {
    const float A = 2.0f / ((g + 1.0f) * K.rho);
    const float B = (g - 1.0f) / (g + 1.0f) * pbK;
    const float sq = sqrtf(A / (pb + B));
    f = dp * sq;
    df = sq * (1.0f - 0.5f * dp / (pb + B));
  } else {
    // (pb/pbK)^a - 1 as expm1(a log1p(dp/pbK)): no cancellation for weak waves
    const float x = dp / pbK;
    const float qm1 = expm1f((g - 1.0f) / (2.0f * g) * log1pf(x));
    f = 2.0f * K.c / (g - 1.0f) * qm1;
    df = (1.0f + qm1) / ((1.0f + x) * K.rho * K.c);
  }
  return true;
}

__device__ inline bool mg_hugoniot_f(const EosP<float>& q, const SideF& K, float p, float& rho_out, float& drdp) {
  float lo = K.rho, hi = q.rho0 * q.s / (q.s - 1.0f);
  if (!(hi > lo)) return false;
  float rho = K.rho + (p - K.p) / (K.c * K.c);
  if (!(rho > lo && rho < hi)) rho = 0.5f * (lo + hi);
  for (int it = 0; it < 40; ++it) {
    const float eta = 1.0f - q.rho0 / rho;
    if (!(eta < q.eta_max)) return false;
    float pR, dpR, eR, deR;
    mg_ref<float>(q, eta, pR, dpR, eR, deR);
    const float e = eR + (p - pR) * q.inv_rg;
    const float ir2 = 1.0f / (rho * rho);
    const float dedr = (deR - dpR * q.inv_rg) * q.rho0 * ir2;
    const float H = e - K.e - 0.5f * (p + K.p) * (1.0f / K.rho - 1.0f / rho);
    const float dH = dedr - 0.5f * (p + K.p) * ir2;
    if (H > 0.0f) lo = rho; else hi = rho;
    float rn = rho - H / dH;
    if (!(rn >= lo && rn <= hi)) rn = 0.5f * (lo + hi);
    const bool conv = fabsf(rn - rho) <= 1e-6f * rn;
    rho = rn;
    if (conv) {
      const float ir = 1.0f / rho;
      mg_ref<float>(q, 1.0f - q.rho0 * ir, pR, dpR, eR, deR);
      const float dedn = (deR - dpR * q.inv_rg) * q.rho0 * ir * ir;
      const float Hp = q.inv_rg - 0.5f * (1.0f / K.rho - ir);
      const float Hr = dedn - 0.5f * (p + K.p) * ir * ir;
      rho_out = rho;
      drdp = -Hp / Hr;
      return true;
    }
  }
  return false;
}

__device__ inline bool mg_rhs_f(const EosP<float>& q, float p, float rho, float& drho, float& dfv) {
  float e, c2;
  if (!eos_e_c2<float>(q, rho, 1.0f / rho, p, e, c2)) return false;
  drho = 1.0f / c2;
  dfv = 1.0f / (rho * sqrtf(c2));
  return true;
}

__device__ inline bool wave_mg_f(const EosP<float>& q, const SideF& K, float p, float& f, float& df) {
  const float dp = p - K.p, z = K.rho * K.c;
  if (fabsf(dp) <= 1e-5f * z * K.c) {  // acoustic start for rounding-level waves
    f = dp / z;
    df = 1.0f / z;
    return true;
  }
  if (p > K.p) {
    float rho, drdp;
    if (!mg_hugoniot_f(q, K, p, rho, drdp)) return false;
    const float dv = 1.0f / K.rho - 1.0f / rho;
    const float fv = sqrtf(dp * dv);
    if (!(fv > 0.0f)) return false;
    f = fv;
    df = (dv + dp * drdp / (rho * rho)) / (2.0f * fv);
    return true;
  }
  float nsd = ceilf((float)kRk4Steps * fabsf(dp) / q.rk4_span);
  nsd = nsd >= 1.0f ? (nsd > (float)kRk4Steps ? (float)kRk4Steps : nsd) : 1.0f;
  const int ns = (int)nsd;
  const float hs = dp / (float)ns;
  float rho = K.rho, fv = 0.0f;
  for (int i = 0; i < ns; ++i) {
    const float pi = K.p + (float)i * hs;
    float k1r, k1f, k2r, k2f, k3r, k3f, k4r, k4f;
    if (!mg_rhs_f(q, pi, rho, k1r, k1f) || !mg_rhs_f(q, pi + 0.5f * hs, rho + 0.5f * hs * k1r, k2r, k2f) ||
        !mg_rhs_f(q, pi + 0.5f * hs, rho + 0.5f * hs * k2r, k3r, k3f) ||
        !mg_rhs_f(q, pi + hs, rho + hs * k3r, k4r, k4f))
      return false;
    rho = rho + hs / 6.0f * (k1r + 2.0f * k2r + 2.0f * k3r + k4r);
    fv = fv + hs / 6.0f * (k1f + 2.0f * k2f + 2.0f * k3f + k4f);
  }
  float e, c2;
  if (!eos_e_c2<float>(q, rho, 1.0f / rho, p, e, c2)) return false;
  f = fv;
  df = 1.0f / (rho * sqrtf(c2));
  return true;
}

// F(p) = f_L + f_R + (u_R - u_L) and its slope on the FP32 curves; false if a
// curve is undefined at p or F is not finite (the caller checks the slope).
__device__ inline bool riemann_F_f(const EosP<float>& qL, const SideF& L, const EosP<float>& qR, const SideF& Rs,
                                   float p, float& F, float& dF) {
  float fL, dfL, fR, dfR;
  const bool okL = qL.type == M2C_EOS_SG ? wave_sg_f(qL, L, p, fL, dfL) : wave_mg_f(qL, L, p, fL, dfL);
  if (!okL) return false;
  const bool okR = qR.type == M2C_EOS_SG ? wave_sg_f(qR, Rs, p, fR, dfR) : wave_mg_f(qR, Rs, p, fR, dfR);
  if (!okR) return false;
  F = fL + fR + (Rs.u - L.u);
  dF = dfL + dfR;
  return isfinite(F);
}

// FP32 Newton on p* from the PVRS guess; false if it fails, signals a vacuum
// or does not reach |dp| <= 1e-5 |p| in 30 steps.
static __device__ __noinline__ bool riemann_newton_f(const EosP<float>& qL, float rl, float ul, float pl, const EosP<float>& qR,
                                        float rr, float ur, float pr, float& p_out, int& iters,
                                        float p_start) {
  // FP32 wave curves exist for the stiffened gas and Mie-Grueneisen only
  if ((qL.type != M2C_EOS_SG && qL.type != M2C_EOS_MG) || (qR.type != M2C_EOS_SG && qR.type != M2C_EOS_MG))
    return false;
  SideF L, Rs;
  if (!make_side_f(qL, rl, ul, pl, L) || !make_side_f(qR, rr, ur, pr, Rs)) return false;
  const float plow = fmaxf(eos_plow_f(qL), eos_plow_f(qR));
  float F, dF;
  if (isfinite(plow)) {
    if (!riemann_F_f(qL, L, qR, Rs, plow, F, dF) || F >= 0.0f) return false;
  }
  float p = 0.5f * (L.p + Rs.p) - 0.125f * (Rs.u - L.u) * (L.rho + Rs.rho) * (L.c + Rs.c);
  if (p_start > plow && p_start < INFINITY) p = p_start;
  if (!(p > plow)) {
    float gap = fminf(L.p, Rs.p) - plow;
    if (!(gap > 0.0f)) gap = fmaxf(L.p, Rs.p) - plow;
    p = plow + 1e-3f * gap;
  }
  for (int it = 1; it <= 30; ++it) {
    if (!riemann_F_f(qL, L, qR, Rs, p, F, dF) || !(dF > 0.0f)) return false;
    float pn = p - F / dF;
    if (!(pn > plow)) pn = 0.5f * (p + plow);
    const bool small = fabsf(pn - p) <= 1e-5f * fabsf(pn);
    p = pn;
    if (small) {
      p_out = p;
      iters = it;
      return true;
    }
  }
  return false;
}

static __device__ __noinline__ int riemann_solve_mixed(const EosP<float>& qLf, const EosDev& qL, double rl, double ul, double pl,
                                          const EosP<float>& qRf, const EosDev& qR, double rr, double ur, double pr,
                                          RiemannOut& out, int& iters,
                                          double p_start = NAN) {
  float p32;
  int it32 = 0;
  Side L, Rs;
  if (riemann_newton_f(qLf, d2f(rl), d2f(ul), d2f(pl), qRf, d2f(rr), d2f(ur), d2f(pr), p32, it32, (float)p_start) &&
      make_side(qL, rl, ul, pl, L) && make_side(qR, rr, ur, pr, Rs)) {
    const double plow = fmax(eos_plow(qL), eos_plow(qR));
    fix_substeps(qL, L, qR, Rs, plow);
    double p = f2d(p32);
    for (int k = 0; k < 2; ++k) {
      double fL, dfL, rL, dL = 0.0, fR, dfR, rR, dR = 0.0;
      if (!(p > plow) || wave(qL, L, p, fL, dfL, rL, true, &dL) || wave(qR, Rs, p, fR, dfR, rR, true, &dR)) break;
      const double F = fL + fR + (Rs.u - L.u), dF = dfL + dfR;
      const double dp = -F / dF;
      // a slope that is not finite (a wave of rounding-level strength on a
      // shock curve) leaves the problem to the FP64 iteration
      if (!(isfinite(dF) && dF > 0.0 && isfinite(dL) && isfinite(dR) && fabs(dp) <= 1e-5 * fabs(p) &&
            p + dp > plow))
        break;
      if (k == 1 || fabs(dp) <= 1e-9 * fabs(p)) {
        out.p = p + dp;
        out.u = 0.5 * (L.u + Rs.u) + 0.5 * (fR - fL) + 0.5 * (dfR - dfL) * dp;
        out.rhoL = rL + dL * dp;
        out.rhoR = rR + dR * dp;
        iters = it32 + 1 + k;
        return M2C_OK;
      }
      p += dp;
    }
  }
  return riemann_solve(qL, rl, ul, pl, qR, rr, ur, pr, out, iters, p_start);
}

}  // namespace m2c
