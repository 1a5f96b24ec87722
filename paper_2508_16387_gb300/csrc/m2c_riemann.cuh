// Exact two-material Riemann solver of the FIVER flux (arXiv 2508.16387,
// Sec. 4.2), FP64 with an optional FP32 start: wave curves of the stiffened
// gas, NASG, Mie-Grueneisen and JWL materials, the Newton iteration on p* and
// the star states. Used by the interface and Riemann kernels of m2c_solver.cu;
// the bulk kernels do not include it.
#pragma once
#include "m2c_physics.cuh"

namespace m2c {

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
  // when u_R - u_L >= 0; no vacuum test with a JWL side (its rarefaction needs
  // p > 0). F increases with p, so a root above p_low found by the Newton
  // iteration implies F(p_low) < 0: the test is made only when the iteration
  // does not converge (before the bisection), which spares each converged
  // problem an evaluation of its curves down to p_low
  const bool vacuum_test = isfinite(plow) && Rs.u - L.u >= 0.0 && qL.type != M2C_EOS_JWL && qR.type != M2C_EOS_JWL;
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
    if (vacuum_test) {
      st = riemann_F(qL, L, qR, Rs, plow, F, dF);
      if (st) return st;
      if (F >= 0.0) return M2C_EVACUUM;
    }
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

// FP32 Newton on p* from the PVRS guess; false if it fails, ends within 1e-4
// of the lowest admissible pressure (where a vacuum would take it) or does not
// reach |dp| <= 1e-5 |p| in 30 steps.
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
  // no vacuum test here (as in the FP64 solve, a root above p_low rules a vacuum
  // out): with a vacuum the iterates only approach p_low, so a "root" within
  // 1e-4 of p_low is rejected and the problem left to the FP64 solve
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
      if (isfinite(plow) && !(p - plow > 1e-4f * fabsf(p))) return false;
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
