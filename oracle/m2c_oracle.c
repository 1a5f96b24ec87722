/*
 * m2c_oracle.c -- plain, slow, CPU FP64 oracle for one time step of the
 * multi-material finite-volume method of M2C (arXiv 2508.16387).
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only callers. The GPU solver shares no
 * code, header, table or helper with this file, and this file includes nothing
 * from it. Build: gcc -O2 -ffp-contract=off [-fopenmp] -shared -fPIC.
 *
 * Every function names the passage of the paper it follows. Where the paper is
 * silent the reading taken is marked "Reading R<n>", numbered as in the
 * design notes. OpenMP is used only over cells whose results are independent
 * of each other, so the result does not depend on the thread count.
 *
 * Beyond the configuration the GPU solver runs (TVD RK2, modified van Albada,
 * HLLC, stiffened gas / Mie-Grueneisen, Cartesian), a grid selects the paper's
 * other choices: TVD RK3 or forward Euler and a constant time step (Sec. 4.3),
 * the MC limiter (App. D), the local Lax-Friedrichs flux (App. C.1), the NASG
 * and JWL equations of state (Sec. 3.3, App. B.2), the spherical and
 * cylindrical forms (Sec. 3.4) and mirror boundaries.
 *
 * Conventions: SI units. State per cell W = (rho, rho u, rho v, rho w, rho E),
 * primitive P = (rho, u, v, w, p). Arrays are structure-of-arrays with x
 * fastest: field f of cell (i,j,k) is a[f*N + (k*ny + j)*nx + i].
 * Material id m = 1 where phi < 0, else 0 (phi = 0 belongs to material 0).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* status codes (their numeric values match the solver library's) */
#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ENOCONV 4
#define OR_ENONPHYS 5
#define OR_EVACUUM 6

#define EOS_SG 0 /* stiffened gas, prm = {gamma, p_c}; p_c = 0 is a perfect gas */
#define EOS_MG 1 /* Mie-Grueneisen, prm = {rho0, c0, s, Gamma0, e0, eta_min} */
#define EOS_NASG 2 /* Noble-Abel stiffened gas, prm = {gamma, p_c, b, e_c} (Sec. 3.3, Eq. NASG_EOS) */
#define EOS_JWL 3  /* Jones-Wilkins-Lee, prm = {omega, A1, A2, R1, R2, rho0} (App. B.2, Eq. JWL_EOS) */

#define BC_TRANSMISSIVE 0
#define BC_PERIODIC 1
#define BC_SYMMETRY 2 /* mirror: ghost cells reflect the interior, the normal velocity negated */

#define GEOM_CARTESIAN 0
#define GEOM_CYLINDRICAL 1 /* x is the radius r, z the axis (Sec. 3.4, Eq. Euler_cylindrical) */
#define GEOM_SPHERICAL 2   /* x is the radius r (Sec. 3.4, Eq. euler1d_spherical) */

/* Riemann solver controls, Reading R6 */
#define NEWTON_TOL 1e-12
#define NEWTON_CAP 50
#define BISECT_CAP 200
#define HUGONIOT_TOL 1e-14
#define HUGONIOT_CAP 100
#define RK4_SUBSTEPS 64      /* substeps of a rarefaction spanning at least RK4_SPAN_FRAC * K0 */
#define RK4_SPAN_FRAC 0.05

typedef struct {
  int type;
  double prm[6];
} or_eos_t;

typedef struct {
  int n[3];
  int bc[6]; /* x-, x+, y-, y+, z-, z+ */
  double h;
  double cfl;
  int reinit_every; /* 0: never */
  int reinit_iters;
  or_eos_t eos[2]; /* eos[0] where phi >= 0, eos[1] where phi < 0 */
  /* scheme options (Sec. 4.3, App. C, App. D); the defaults are the paper's
   * workload choices used everywhere else in this file */
  int rk;          /* Runge-Kutta order: 2 (default), 3 (TVD RK3), 1 (forward Euler) */
  int limiter;     /* LIM_VA_MOD (default) or LIM_MC */
  int flux;        /* FLUX_HLLC (default) or FLUX_LLF */
  double mc_alpha; /* alpha of the MC limiter (1.2 by default) */
  double dt_fixed; /* > 0: constant time step instead of the CFL rule */
  int geom;        /* GEOM_CARTESIAN (default), GEOM_CYLINDRICAL or GEOM_SPHERICAL */
  double x0;       /* lower x coordinate: the radius of the first cell's lower face */
  double band_beta, band_gamma; /* narrow-band level set: tube radii in cells (gamma = 0: full domain) */
} or_grid_t;

#define LIM_VA_MOD 0 /* modified van Albada, App. D */
#define LIM_MC 1     /* monotonized central, App. D, Eq. theta */
#define FLUX_HLLC 0  /* App. C.4 */
#define FLUX_LLF 1   /* local Lax-Friedrichs, App. C.1, Eq. Lax-Friedrichs */

typedef struct {
  double dt;             /* time step of the last step */
  long interface_faces;  /* faces with different materials on the two sides, stage 1 of the last step */
  long newton_max;       /* largest Riemann iteration count seen */
  long flipped;          /* cells that changed material in the last step */
  long err_cell;         /* cell of the first error, -1 if none */
} or_stats_t;

/* ------------------------------------------------------------------ */
/* Equations of state                                                 */
/* ------------------------------------------------------------------ */

/* Mie-Grueneisen reference curves p_R(eta), e_R(eta) and their eta-derivatives,
 * App. B.3: compression (eta > 0), tension down to eta_min, and below eta_min.
 * Reading R1: the "p_H" in e_R of the compression branch is p_R. Reading R4:
 * e0 is a parameter (0 in the workloads). */
static void mg_ref(const or_eos_t* q, double eta, double* pR, double* dpR, double* eR, double* deR) {
  const double rho0 = q->prm[0], c0 = q->prm[1], s = q->prm[2], e0 = q->prm[4], eta_min = q->prm[5];
  const double K0 = rho0 * c0 * c0;
  if (eta > 0.0) {
    double d = 1.0 - s * eta;
    *pR = K0 * eta / (d * d);
    *dpR = K0 * (1.0 + s * eta) / (d * d * d);
    *eR = (*pR) * eta / (2.0 * rho0) + e0;
    *deR = ((*dpR) * eta + (*pR)) / (2.0 * rho0);
  } else if (eta >= eta_min) {
    *pR = K0 * eta;
    *dpR = K0;
    *eR = K0 * eta * eta / (2.0 * rho0) + e0;
    *deR = K0 * eta / rho0;
  } else {
    double pmin = K0 * eta_min;
    *pR = pmin;
    *dpR = 0.0;
    *eR = K0 * eta_min * eta_min / (2.0 * rho0) + e0 + pmin / rho0 * (eta - eta_min);
    *deR = pmin / rho0;
  }
}

/* MG is defined for eta < 1/s (Reading R5: p_R has a pole at eta = 1/s). */
static int mg_eta(const or_eos_t* q, double rho, double* eta) {
  if (!(rho > 0.0)) return OR_ENONPHYS;
  *eta = 1.0 - q->prm[0] / rho;
  if (!(*eta < 1.0 / q->prm[2])) return OR_ENONPHYS;
  return OR_OK;
}

/* JWL (App. B.2, Eq. JWL_EOS): p = omega rho e + f(rho) with
 * f = sum_i A_i (1 - omega rho/(R_i rho0)) exp(-R_i rho0/rho). Reading R35: the
 * first exponential, printed with a plus sign, has the minus sign of the
 * second one and of the temperature law printed with it (with a plus sign the
 * pressure would grow without bound as rho -> 0). f and df/drho. */
static void jwl_f(const or_eos_t* q, double rho, double* f, double* df) {
  double w = q->prm[0], rho0 = q->prm[5];
  *f = 0.0;
  *df = 0.0;
  for (int i = 0; i < 2; ++i) {
    double A = q->prm[1 + i], R = q->prm[3 + i];
    double x = R * rho0 / rho, ex = exp(-x), a = 1.0 - w * rho / (R * rho0);
    *f += A * a * ex;
    *df += A * ex * (-w / (R * rho0) + a * x / rho);
  }
}

/* p(rho, e): NASG with b = e_c = 0 (Sec. 3.3, Eq. NASG_EOS), the full NASG
 * p = (gamma - 1) rho (e - e_c)/(1 - rho b) - gamma p_c (defined for rho b < 1),
 * or MG (App. B.3). */
static int eos_p(const or_eos_t* q, double rho, double e, double* p) {
  if (!(rho > 0.0)) return OR_ENONPHYS;
  if (q->type == EOS_SG) {
    double g = q->prm[0], pc = q->prm[1];
    *p = (g - 1.0) * rho * e - g * pc;
    return OR_OK;
  }
  if (q->type == EOS_NASG) {
    double g = q->prm[0], pc = q->prm[1], b = q->prm[2], ec = q->prm[3];
    if (!(1.0 - rho * b > 0.0)) return OR_ENONPHYS;
    *p = (g - 1.0) * rho * (e - ec) / (1.0 - rho * b) - g * pc;
    return OR_OK;
  }
  if (q->type == EOS_JWL) {
    double f, df;
    jwl_f(q, rho, &f, &df);
    *p = q->prm[0] * rho * e + f;
    return OR_OK;
  }
  double eta, pR, dpR, eR, deR;
  int st = mg_eta(q, rho, &eta);
  if (st) return st;
  mg_ref(q, eta, &pR, &dpR, &eR, &deR);
  *p = pR + q->prm[0] * q->prm[3] * (e - eR);
  return OR_OK;
}

/* e(rho, p): the same relations solved for e. */
static int eos_e(const or_eos_t* q, double rho, double p, double* e) {
  if (!(rho > 0.0)) return OR_ENONPHYS;
  if (q->type == EOS_SG) {
    double g = q->prm[0], pc = q->prm[1];
    *e = (p + g * pc) / ((g - 1.0) * rho);
    return OR_OK;
  }
  if (q->type == EOS_NASG) {
    double g = q->prm[0], pc = q->prm[1], b = q->prm[2], ec = q->prm[3];
    if (!(1.0 - rho * b > 0.0)) return OR_ENONPHYS;
    *e = ec + (p + g * pc) * (1.0 - rho * b) / ((g - 1.0) * rho);
    return OR_OK;
  }
  if (q->type == EOS_JWL) {
    double f, df;
    jwl_f(q, rho, &f, &df);
    *e = (p - f) / (q->prm[0] * rho);
    return OR_OK;
  }
  double eta, pR, dpR, eR, deR;
  int st = mg_eta(q, rho, &eta);
  if (st) return st;
  mg_ref(q, eta, &pR, &dpR, &eR, &deR);
  *e = eR + (p - pR) / (q->prm[0] * q->prm[3]);
  return OR_OK;
}

/* c^2 = dp/drho|_e + (p/rho^2) dp/de|_rho (App. C.2, speed of sound).
 * SG: gamma (p + p_c) / rho. MG: dp/drho|_e = (p_R' - rho0 Gamma0 e_R') rho0/rho^2 and
 * dp/de|_rho = rho0 Gamma0 (Reading R2: the Grueneisen coefficient rho0 Gamma0 is constant). */
static int eos_c2(const or_eos_t* q, double rho, double p, double* c2) {
  if (!(rho > 0.0)) return OR_ENONPHYS;
  if (q->type == EOS_SG) {
    double g = q->prm[0], pc = q->prm[1];
    *c2 = g * (p + pc) / rho;
  } else if (q->type == EOS_NASG) {
    /* dp/drho|_e = (p + gamma p_c)/(rho (1 - rho b)), dp/de|_rho = (gamma - 1) rho/(1 - rho b) */
    double g = q->prm[0], pc = q->prm[1], b = q->prm[2];
    if (!(1.0 - rho * b > 0.0)) return OR_ENONPHYS;
    *c2 = g * (p + pc) / (rho * (1.0 - rho * b));
  } else if (q->type == EOS_JWL) {
    /* dp/drho|_e = omega e + f'(rho) with omega e = (p - f)/rho, dp/de|_rho = omega rho */
    double f, df;
    jwl_f(q, rho, &f, &df);
    *c2 = ((1.0 + q->prm[0]) * p - f) / rho + df;
  } else {
    double eta, pR, dpR, eR, deR;
    int st = mg_eta(q, rho, &eta);
    if (st) return st;
    mg_ref(q, eta, &pR, &dpR, &eR, &deR);
    double rg = q->prm[0] * q->prm[3];
    *c2 = (dpR - rg * deR) * q->prm[0] / (rho * rho) + p * rg / (rho * rho);
  }
  if (!(*c2 > 0.0) || !isfinite(*c2)) return OR_ENONPHYS;
  return OR_OK;
}

/* Lowest admissible pressure on a side: SG needs p + p_c > 0; MG with a
 * finite tensile cutoff has p_min = K0 eta_min, else no bound. */
static double eos_plow(const or_eos_t* q) {
  if (q->type == EOS_SG || q->type == EOS_NASG) return -q->prm[1];
  if (q->type == EOS_JWL) return 0.0; /* Reading R36 */
  if (isfinite(q->prm[5])) return q->prm[0] * q->prm[1] * q->prm[1] * q->prm[5];
  return -INFINITY;
}

/* dp/de|_rho and de/drho|_p of MG at (rho, p), used by the Hugoniot root. */
static int mg_de_drho_p(const or_eos_t* q, double rho, double* de_drho) {
  double eta, pR, dpR, eR, deR;
  int st = mg_eta(q, rho, &eta);
  if (st) return st;
  mg_ref(q, eta, &pR, &dpR, &eR, &deR);
  double rg = q->prm[0] * q->prm[3];
  *de_drho = (deR - dpR / rg) * q->prm[0] / (rho * rho);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Exact two-material Riemann problem, Sec. 4.2 (Eq. 1DRiemannProblem)  */
/* with the interface conditions of Sec. 3.5.1 (Eq. interface_cond)     */
/* ------------------------------------------------------------------ */

typedef struct {
  double rho, u, p, c, e;
  int nrk; /* RK4 substeps of this side's rarefaction curve fixed for one Riemann
            * problem (Reading R6); 0: chosen per evaluation from |p - p_K| */
  double dnode; /* MG: spacing of the fixed RK4 nodes p_K - i dnode of the problem (> 0), 0: none */
} side_t;

/* Wave curve of one side: velocity change f_K(p) across the K-wave that takes
 * the side state to pressure p, its derivative, and the density behind it.
 * SG/PG: the textbook ideal-gas shock and rarefaction relations written in
 * p + p_c (Reading R6). */
static int wave_sg(const or_eos_t* q, const side_t* K, double p, double* f, double* df, double* rs) {
  double g = q->prm[0], pc = q->prm[1];
  double pb = p + pc, pbK = K->p + pc;
  if (!(pb >= 0.0) || !(pbK > 0.0)) return OR_ENONPHYS;
  if (p > K->p) {
    double A = 2.0 / ((g + 1.0) * K->rho);
    double B = (g - 1.0) / (g + 1.0) * pbK;
    double sq = sqrt(A / (pb + B));
    *f = (p - K->p) * sq;
    *df = sq * (1.0 - 0.5 * (p - K->p) / (pb + B));
    double r = pb / pbK, gm = (g - 1.0) / (g + 1.0);
    *rs = K->rho * (r + gm) / (gm * r + 1.0);
  } else {
    double r = pb / pbK;
    *f = 2.0 * K->c / (g - 1.0) * (pow(r, (g - 1.0) / (2.0 * g)) - 1.0);
    *df = pow(r, -(g + 1.0) / (2.0 * g)) / (K->rho * K->c);
    *rs = K->rho * pow(r, 1.0 / g);
  }
  return OR_OK;
}

/* MG shock: density on the Hugoniot through (rho_K, p_K, e_K) at pressure p,
 * H(rho) = e(rho,p) - e_K - (p + p_K)/2 (1/rho_K - 1/rho) = 0 on (rho_K, rho0 s/(s-1)),
 * by Newton's method kept inside a shrinking bracket, stopped at the first step
 * below 1e-14 rho (Reading R6). */
static int mg_hugoniot_rho(const or_eos_t* q, const side_t* K, double p, double* rho_out, double* drho_dp) {
  const double rho0 = q->prm[0], s = q->prm[2], rg = q->prm[0] * q->prm[3];
  double lo = K->rho, hi = rho0 * s / (s - 1.0);
  if (!(hi > lo)) return OR_ENONPHYS;
  double rho = K->rho + (p - K->p) / (K->c * K->c);
  if (!(rho > lo && rho < hi)) rho = 0.5 * (lo + hi);
  int done = 0;
  for (int it = 0; it < HUGONIOT_CAP; ++it) {
    double e, dedr;
    int st = eos_e(q, rho, p, &e);
    if (!st) st = mg_de_drho_p(q, rho, &dedr);
    if (st) return st;
    double H = e - K->e - 0.5 * (p + K->p) * (1.0 / K->rho - 1.0 / rho);
    double dH = dedr - 0.5 * (p + K->p) / (rho * rho);
    if (H > 0.0) lo = rho; else hi = rho;
    double rn = rho - H / dH;
    if (!(rn >= lo && rn <= hi)) rn = 0.5 * (lo + hi);
    int conv = fabs(rn - rho) <= HUGONIOT_TOL * rn;
    rho = rn;
    if (conv) { done = 1; break; }
  }
  if (!done) return OR_ENOCONV;
  /* d rho / dp along the Hugoniot by implicit differentiation of H */
  double dedr;
  int st = mg_de_drho_p(q, rho, &dedr);
  if (st) return st;
  double Hp = 1.0 / rg - 0.5 * (1.0 / K->rho - 1.0 / rho);
  double Hr = dedr - 0.5 * (p + K->p) / (rho * rho);
  *rho_out = rho;
  *drho_dp = -Hp / Hr;
  return OR_OK;
}

/* Right-hand side of the isentrope ODE in p: d rho/dp = 1/c^2, d f/dp = 1/(rho c). */
static int mg_isentrope_rhs(const or_eos_t* q, double p, double rho, double* drho, double* dfv) {
  double c2;
  int st = eos_c2(q, rho, p, &c2);
  if (st) return st;
  *drho = 1.0 / c2;
  *dfv = 1.0 / (rho * sqrt(c2));
  return OR_OK;
}

/* Substeps of the RK4 isentrope integration over a pressure span dp (Reading
 * R6): 64 equal substeps when the span is at least 5% of the reference bulk
 * modulus K0 = rho0 c0^2, proportionally fewer (at least one) for weaker waves,
 * so the substep length never exceeds 0.05 K0 / 64. Within one Riemann problem
 * the count is fixed before the iteration from a bound of the span (see
 * rarefaction_substeps), so that the wave curve is a smooth function of p. */
static int rk4_substeps(const or_eos_t* q, double dp) {
  double K0 = q->prm[0] * q->prm[1] * q->prm[1];
  double n = ceil(RK4_SUBSTEPS * fabs(dp) / (RK4_SPAN_FRAC * K0));
  if (!(n >= 1.0)) n = 1.0;
  if (n > RK4_SUBSTEPS) n = RK4_SUBSTEPS;
  return (int)n;
}

/* One classical RK4 substep of the isentrope (rho, f) from pressure pi by hs. */
static int mg_rk4_substep(const or_eos_t* q, double pi, double hs, double* rho, double* fv) {
  double k1r, k1f, k2r, k2f, k3r, k3f, k4r, k4f;
  int st = mg_isentrope_rhs(q, pi, *rho, &k1r, &k1f);
  if (!st) st = mg_isentrope_rhs(q, pi + 0.5 * hs, *rho + 0.5 * hs * k1r, &k2r, &k2f);
  if (!st) st = mg_isentrope_rhs(q, pi + 0.5 * hs, *rho + 0.5 * hs * k2r, &k3r, &k3f);
  if (!st) st = mg_isentrope_rhs(q, pi + hs, *rho + hs * k3r, &k4r, &k4f);
  if (st) return st;
  *rho = *rho + hs / 6.0 * (k1r + 2.0 * k2r + 2.0 * k3r + k4r);
  *fv = *fv + hs / 6.0 * (k1f + 2.0 * k2f + 2.0 * k3f + k4f);
  return OR_OK;
}

/* MG wave curve. Shock: f = sqrt((p - p_K)(1/rho_K - 1/rho_H(p))). Rarefaction:
 * f = integral from p_K to p of dp/(rho c) along the isentrope, integrated
 * together with rho by classical RK4 in p (Reading R6): inside a Riemann
 * problem, on the fixed nodes p_K - i dnode of the problem (dnode = the span
 * bound over the substep count), full substeps down to the last node above p
 * and a partial one to p, so that the curve is continuous and smooth in p (its
 * slope jumps at a node only by the RK4 truncation error) and evaluations at
 * nearby pressures share their nodes; beyond the span bound, and for a wave
 * evaluated alone, equal substeps over p_K - p. */
static int wave_mg(const or_eos_t* q, const side_t* K, double p, double* f, double* df, double* rs) {
  if (p == K->p) {
    *f = 0.0;
    *df = 1.0 / (K->rho * K->c);
    *rs = K->rho;
    return OR_OK;
  }
  if (p > K->p) {
    double rho, drdp;
    int st = mg_hugoniot_rho(q, K, p, &rho, &drdp);
    if (st) return st;
    double dv = 1.0 / K->rho - 1.0 / rho;
    double fv = sqrt((p - K->p) * dv);
    *f = fv;
    *df = (dv + (p - K->p) * drdp / (rho * rho)) / (2.0 * fv);
    *rs = rho;
    return OR_OK;
  }
  double rho = K->rho, fv = 0.0;
  double dp = K->p - p;
  if (K->dnode > 0.0 && dp < K->nrk * K->dnode) {
    /* inside the problem's span bound: m full substeps on the fixed nodes p_K - i dnode,
     * then one partial substep from the last node to p (Reading R6) */
    int m = (int)floor(dp / K->dnode);
    if (m > K->nrk - 1) m = K->nrk - 1;
    for (int i = 0; i < m; ++i) {
      int st = mg_rk4_substep(q, K->p - i * K->dnode, -K->dnode, &rho, &fv);
      if (st) return st;
    }
    double hp = dp - m * K->dnode;
    if (hp > 0.0) {
      int st = mg_rk4_substep(q, K->p - m * K->dnode, -hp, &rho, &fv);
      if (st) return st;
    }
  } else {
    int ns = K->nrk > 0 ? K->nrk : rk4_substeps(q, p - K->p);
    double hs = (p - K->p) / ns;
    for (int i = 0; i < ns; ++i) {
      int st = mg_rk4_substep(q, K->p + i * hs, hs, &rho, &fv);
      if (st) return st;
    }
  }
  double c2;
  int st = eos_c2(q, rho, p, &c2);
  if (st) return st;
  *f = fv;
  *df = 1.0 / (rho * sqrt(c2));
  *rs = rho;
  return OR_OK;
}

/* JWL Hugoniot through K at pressure p > p_K: the root of
 * H(rho) = e(rho, p) - e_K - (p + p_K)(1/rho_K - 1/rho)/2 with rho > rho_K, by
 * Newton safeguarded in a bracket [rho_K, rho_hi] (H(rho_K) > 0; rho_hi starts
 * at the strong-shock compression rho_K (omega + 2)/omega of a gas with
 * Grueneisen coefficient omega and doubles until H(rho_hi) < 0), the same
 * tolerance and stopping rule as the MG root; d rho/dp by implicit
 * differentiation. de/drho|_p = -(f'(rho) + omega e)/(omega rho). */
static int jwl_hugoniot_rho(const or_eos_t* q, const side_t* K, double p, double* rho_out, double* drho_dp) {
  double w = q->prm[0];
  double lo = K->rho, hi = K->rho * (w + 2.0) / w;
  int bracketed = 0;
  for (int k = 0; k < 60 && !bracketed; ++k) {
    double e;
    int st = eos_e(q, hi, p, &e);
    if (st) return st;
    if (e - K->e - 0.5 * (p + K->p) * (1.0 / K->rho - 1.0 / hi) < 0.0) bracketed = 1;
    else { lo = hi; hi = 2.0 * hi; }
  }
  if (!bracketed) return OR_ENOCONV;
  double rho = K->rho + (p - K->p) / (K->c * K->c);
  if (!(rho > lo && rho < hi)) rho = 0.5 * (lo + hi);
  int done = 0;
  for (int it = 0; it < HUGONIOT_CAP; ++it) {
    double e, f, df;
    int st = eos_e(q, rho, p, &e);
    if (st) return st;
    jwl_f(q, rho, &f, &df);
    double dedr = -(df + w * e) / (w * rho);
    double H = e - K->e - 0.5 * (p + K->p) * (1.0 / K->rho - 1.0 / rho);
    double dH = dedr - 0.5 * (p + K->p) / (rho * rho);
    if (H > 0.0) lo = rho; else hi = rho;
    double rn = rho - H / dH;
    if (!(rn >= lo && rn <= hi)) rn = 0.5 * (lo + hi);
    int conv = fabs(rn - rho) <= HUGONIOT_TOL * rn;
    rho = rn;
    if (conv) { done = 1; break; }
  }
  if (!done) return OR_ENOCONV;
  double e, f, df;
  int st = eos_e(q, rho, p, &e);
  if (st) return st;
  jwl_f(q, rho, &f, &df);
  double Hp = 1.0 / (w * rho) - 0.5 * (1.0 / K->rho - 1.0 / rho);
  double Hr = -(df + w * e) / (w * rho) - 0.5 * (p + K->p) / (rho * rho);
  *rho_out = rho;
  *drho_dp = -Hp / Hr;
  return OR_OK;
}

/* JWL wave curve. Shock: f = sqrt((p - p_K)(1/rho_K - 1/rho_H(p))). Rarefaction
 * (Reading R36): the isentrope d rho/dp = 1/c^2, df/dp = 1/(rho c) integrated by
 * classical RK4 in s = ln p (d rho/ds = p/c^2, df/ds = p/(rho c)) on equal
 * substeps, 256 per unit of |ln(p/p_K)| and at least 8 (relative error about
 * 1e-12 over five decades), since detonation products expand over decades of
 * pressure; it needs p > 0. */
static int wave_jwl(const or_eos_t* q, const side_t* K, double p, double* f, double* df, double* rs) {
  if (p == K->p) {
    *f = 0.0;
    *df = 1.0 / (K->rho * K->c);
    *rs = K->rho;
    return OR_OK;
  }
  if (p > K->p) {
    double rho, drdp;
    int st = jwl_hugoniot_rho(q, K, p, &rho, &drdp);
    if (st) return st;
    double dv = 1.0 / K->rho - 1.0 / rho;
    double fv = sqrt((p - K->p) * dv);
    *f = fv;
    *df = (dv + (p - K->p) * drdp / (rho * rho)) / (2.0 * fv);
    *rs = rho;
    return OR_OK;
  }
  if (!(p > 0.0) || !(K->p > 0.0)) return OR_ENONPHYS;
  double span = log(p / K->p);
  double nd = ceil(256.0 * fabs(span));
  int ns = K->nrk > 0 ? K->nrk : (nd < 8.0 ? 8 : (int)nd);
  double hs = span / ns, s0 = log(K->p);
  double rho = K->rho, fv = 0.0;
  for (int i = 0; i < ns; ++i) {
    double si = s0 + i * hs;
    double k1r, k1f, k2r, k2f, k3r, k3f, k4r, k4f, pp, c2;
    int st;
    pp = exp(si);
    st = eos_c2(q, rho, pp, &c2);
    if (st) return st;
    k1r = pp / c2; k1f = pp / (rho * sqrt(c2));
    pp = exp(si + 0.5 * hs);
    double r2 = rho + 0.5 * hs * k1r;
    st = eos_c2(q, r2, pp, &c2);
    if (st) return st;
    k2r = pp / c2; k2f = pp / (r2 * sqrt(c2));
    double r3 = rho + 0.5 * hs * k2r;
    st = eos_c2(q, r3, pp, &c2);
    if (st) return st;
    k3r = pp / c2; k3f = pp / (r3 * sqrt(c2));
    pp = exp(si + hs);
    double r4 = rho + hs * k3r;
    st = eos_c2(q, r4, pp, &c2);
    if (st) return st;
    k4r = pp / c2; k4f = pp / (r4 * sqrt(c2));
    rho = rho + hs / 6.0 * (k1r + 2.0 * k2r + 2.0 * k3r + k4r);
    fv = fv + hs / 6.0 * (k1f + 2.0 * k2f + 2.0 * k3f + k4f);
  }
  double c2;
  int st = eos_c2(q, rho, p, &c2);
  if (st) return st;
  *f = fv;
  *df = 1.0 / (rho * sqrt(c2));
  *rs = rho;
  return OR_OK;
}

/* NASG wave curves in P = p + p_c and the covolume-reduced specific volume
 * w = 1/rho - b. Shock: the Hugoniot energy equation e - e_K = (p + p_K)(1/rho_K
 * - 1/rho)/2 is linear in w and gives w = w_K (gm r + 1)/(r + gm), r = P/P_K,
 * gm = (gamma - 1)/(gamma + 1), so f = (p - p_K) sqrt(A/(P + gm P_K)) with
 * A = 2 w_K/(gamma + 1). Rarefaction: the isentrope P w^gamma = const gives
 * rho c = sqrt(gamma P/w), and the integral of dp/(rho c) is
 * f = 2 c_K (1 - b rho_K)/(gamma - 1) (r^((gamma-1)/(2 gamma)) - 1). With b = 0
 * both are the stiffened-gas curves of wave_sg. */
static int wave_nasg(const or_eos_t* q, const side_t* K, double p, double* f, double* df, double* rs) {
  double g = q->prm[0], pc = q->prm[1], b = q->prm[2];
  double P = p + pc, PK = K->p + pc;
  double wK = 1.0 / K->rho - b;
  if (!(P >= 0.0) || !(PK > 0.0) || !(wK > 0.0)) return OR_ENONPHYS;
  double r = P / PK;
  if (p > K->p) {
    double gm = (g - 1.0) / (g + 1.0);
    double A = 2.0 * wK / (g + 1.0);
    double D = P + gm * PK;
    double sq = sqrt(A / D);
    *f = (p - K->p) * sq;
    *df = sq * (1.0 - 0.5 * (p - K->p) / D);
    *rs = 1.0 / (b + wK * (gm * r + 1.0) / (r + gm));
  } else {
    *f = 2.0 * K->c * (1.0 - b * K->rho) / (g - 1.0) * (pow(r, (g - 1.0) / (2.0 * g)) - 1.0);
    double w = wK * pow(r, -1.0 / g);
    *df = sqrt(w / (g * P));
    *rs = 1.0 / (b + w);
  }
  return OR_OK;
}

static int wave(const or_eos_t* q, const side_t* K, double p, double* f, double* df, double* rs) {
  if (q->type == EOS_SG) return wave_sg(q, K, p, f, df, rs);
  if (q->type == EOS_NASG) return wave_nasg(q, K, p, f, df, rs);
  if (q->type == EOS_JWL) return wave_jwl(q, K, p, f, df, rs);
  return wave_mg(q, K, p, f, df, rs);
}

static int make_side(const or_eos_t* q, const double w[3], side_t* K) {
  K->rho = w[0];
  K->u = w[1];
  K->p = w[2];
  K->nrk = 0;
  K->dnode = 0.0;
  double c2;
  int st = eos_c2(q, K->rho, K->p, &c2);
  if (st) return st;
  K->c = sqrt(c2);
  return eos_e(q, K->rho, K->p, &K->e);
}

/* Reading R6: within one Riemann problem the substep count of side K's
 * rarefaction curve is fixed before the iteration (so that every evaluation
 * lies on one smooth curve of p) from an upper bound of the pressure drop
 * across it. The star pressure is at least p_lo = max(p_low, min(p_J, p_ac))
 * with p_ac = (Z_R p_L + Z_L p_R - Z_L Z_R (u_R - u_L))/(Z_L + Z_R), Z = rho c:
 * if the other side J carries a shock, p* > p_J; if it carries a rarefaction
 * too, each rarefaction curve lies below its acoustic tangent,
 * |f_K(p)| >= |p - p_K|/Z_K (rho c falls along an isentrope as p falls), and
 * F(p*) = 0 then gives p* >= p_ac. MG: the count of rk4_substeps for the span
 * p_K - p_lo, and the node spacing span / count of the fixed RK4 nodes. JWL: 256 per unit of ln(p_K/p_lo) and at least 8, with p_lo
 * kept at or above 1e-6 p_K. Other EOS: closed forms, no substeps. */
static void set_rarefaction_steps(const or_eos_t* q, side_t* K, double p_lo) {
  if (q->type == EOS_MG) {
    double span = fmax(K->p - p_lo, 0.0);
    K->nrk = rk4_substeps(q, span);
    K->dnode = 0.0;
    if (span > 0.0 && isfinite(span)) K->dnode = span / K->nrk;
  } else if (q->type == EOS_JWL) {
    double lo = fmax(p_lo, 1e-6 * K->p);
    double nd = ceil(256.0 * log(K->p / lo));
    K->nrk = nd < 8.0 ? 8 : (int)nd;
  }
}

/* F(p) = f_L(p) + f_R(p) + (u_R - u_L), increasing in p. */
static int riemann_F(const or_eos_t* qL, const side_t* L, const or_eos_t* qR, const side_t* R, double p, double* F, double* dF) {
  double fL, dfL, rL, fR, dfR, rR;
  int st = wave(qL, L, p, &fL, &dfL, &rL);
  if (!st) st = wave(qR, R, p, &fR, &dfR, &rR);
  if (st) return st;
  *F = fL + fR + (R->u - L->u);
  *dF = dfL + dfR;
  return OR_OK;
}

/* Exact solution of the 1D two-material Riemann problem: the star pressure p*
 * solves F(p*) = 0 (Newton from the PVRS guess, kept above the lowest
 * admissible pressure; stop at the first step with |dp| <= 1e-12 |p|, whose
 * update leaves an error of the order of that step squared (Reading R6); after
 * 50 steps, bisection). u* = (u_L + u_R)/2 + (f_R - f_L)/2; rho*_K from the
 * K-wave. Reading R7: no vacuum solution is built; if F(p_low) >= 0 the call
 * fails with OR_EVACUUM. Both wave curves increase with p and vanish at their
 * side's pressure (>= p_low), so F(p_low) <= u_R - u_L: the test is only made
 * when u_R - u_L >= 0; and since F increases with p, a root above p_low found
 * by Newton rules a vacuum out, so the test is made only when Newton has not
 * converged (before the bisection). This also keeps a solution whose wave
 * curves cannot be evaluated at p_low itself: the MG isentrope's sound speed
 * vanishes at the tensile cutoff p_min = K0 eta_min. out = {p*, u*, rho*_L,
 * rho*_R}. */
static int riemann(const or_eos_t* qL, const double wL[3], const or_eos_t* qR, const double wR[3], double out[4], int* iters) {
  side_t L, R;
  int st = make_side(qL, wL, &L);
  if (!st) st = make_side(qR, wR, &R);
  if (st) return st;
  double plow = fmax(eos_plow(qL), eos_plow(qR));
  double ZL = L.rho * L.c, ZR = R.rho * R.c;
  double pac = (ZR * L.p + ZL * R.p - ZL * ZR * (R.u - L.u)) / (ZL + ZR);
  set_rarefaction_steps(qL, &L, fmax(plow, fmin(R.p, pac)));
  set_rarefaction_steps(qR, &R, fmax(plow, fmin(L.p, pac)));
  double F, dF;
  /* Reading R36: no vacuum test with a JWL side (its rarefaction needs p > 0) */
  const int vacuum_test = isfinite(plow) && R.u - L.u >= 0.0 && qL->type != EOS_JWL && qR->type != EOS_JWL;
  double p = 0.5 * (L.p + R.p) - 0.125 * (R.u - L.u) * (L.rho + R.rho) * (L.c + R.c);
  if (!(p > plow)) {
    double gap = fmin(L.p, R.p) - plow;
    if (!(gap > 0.0)) gap = fmax(L.p, R.p) - plow;
    p = plow + 1e-3 * gap;
  }
  int it = 0, conv = 0;
  for (it = 1; it <= NEWTON_CAP; ++it) {
    st = riemann_F(qL, &L, qR, &R, p, &F, &dF);
    if (st) return st;
    double pn = p - F / dF;
    if (!(pn > plow)) pn = 0.5 * (p + plow);
    int small = fabs(pn - p) <= NEWTON_TOL * fabs(pn);
    p = pn;
    if (small) { conv = 1; break; }
  }
  if (!conv) {
    if (vacuum_test) {
      st = riemann_F(qL, &L, qR, &R, plow, &F, &dF);
      if (st) return st;
      if (F >= 0.0) return OR_EVACUUM;
    }
    /* bisection on a bracket [a, b] with F(a) < 0 < F(b) */
    double a = plow, b = fmax(L.p, R.p);
    if (!isfinite(a)) {
      a = fmin(L.p, R.p);
      for (int k = 0; k < BISECT_CAP; ++k) {
        st = riemann_F(qL, &L, qR, &R, a, &F, &dF);
        if (st) return st;
        if (F < 0.0) break;
        a = a - 2.0 * fabs(a) - 1.0;
      }
    }
    for (int k = 0; k < BISECT_CAP; ++k) {
      st = riemann_F(qL, &L, qR, &R, b, &F, &dF);
      if (st) return st;
      if (F > 0.0) break;
      b = 2.0 * b + fabs(b) + 1.0;
    }
    int ok = 0;
    for (int k = 0; k < BISECT_CAP; ++k) {
      double m = 0.5 * (a + b);
      st = riemann_F(qL, &L, qR, &R, m, &F, &dF);
      if (st) return st;
      if (F < 0.0) a = m; else b = m;
      ++it;
      if (b - a <= 1e-14 * fmax(fabs(a), fabs(b))) { ok = 1; break; }
    }
    if (!ok) return OR_ENOCONV;
    p = 0.5 * (a + b);
  }
  double fL, dfL, rL, fR, dfR, rR;
  st = wave(qL, &L, p, &fL, &dfL, &rL);
  if (!st) st = wave(qR, &R, p, &fR, &dfR, &rR);
  if (st) return st;
  out[0] = p;
  out[1] = 0.5 * (L.u + R.u) + 0.5 * (fR - fL);
  out[2] = rL;
  out[3] = rR;
  if (iters) *iters = it;
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* HLLC flux, App. C.4                                                  */
/* ------------------------------------------------------------------ */

/* Physical flux F(W).n for n = e_d, Sec. 3.2 (Eq. NSEquation_terms). */
static void phys_flux(const double P[5], double E, int d, double F[5]) {
  double rho = P[0], un = P[1 + d], p = P[4];
  F[0] = rho * un;
  F[1] = rho * un * P[1];
  F[2] = rho * un * P[2];
  F[3] = rho * un * P[3];
  F[1 + d] += p;
  F[4] = (rho * E + p) * un;
}

/* HLLC with the wave-speed estimates S_L = min(u_L - c_L, u_R - c_R),
 * S_R = max(u_L + c_L, u_R + c_R) and the contact speed S* as printed.
 * Star state W*_K = rho_K (S_K - u_K)/(S_K - S*) [1, V*, E*_K] with the normal
 * velocity S* and the tangential velocity of side K. Reading R13: E*_K =
 * E_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K))), E per unit mass.
 * Inputs are primitive states; one EOS for the whole face (Reading R15). */
static int hllc(const or_eos_t* q, const double Lp[5], const double Rp[5], int d, double F[5]) {
  double c2L, c2R, eL, eR;
  int st = eos_c2(q, Lp[0], Lp[4], &c2L);
  if (!st) st = eos_c2(q, Rp[0], Rp[4], &c2R);
  if (!st) st = eos_e(q, Lp[0], Lp[4], &eL);
  if (!st) st = eos_e(q, Rp[0], Rp[4], &eR);
  if (st) return st;
  double cL = sqrt(c2L), cR = sqrt(c2R);
  double rL = Lp[0], uL = Lp[1 + d], pL = Lp[4];
  double rR = Rp[0], uR = Rp[1 + d], pR = Rp[4];
  double EL = eL + 0.5 * ((Lp[1] * Lp[1] + Lp[2] * Lp[2]) + Lp[3] * Lp[3]);
  double ER = eR + 0.5 * ((Rp[1] * Rp[1] + Rp[2] * Rp[2]) + Rp[3] * Rp[3]);
  double SL = fmin(uL - cL, uR - cR);
  double SR = fmax(uL + cL, uR + cR);
  double Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
  const double* K;
  double EK, SK;
  if (0.0 <= SL) {
    phys_flux(Lp, EL, d, F);
    return OR_OK;
  } else if (0.0 <= Ss) {
    K = Lp; EK = EL; SK = SL;
  } else if (0.0 <= SR) {
    K = Rp; EK = ER; SK = SR;
  } else {
    phys_flux(Rp, ER, d, F);
    return OR_OK;
  }
  double FK[5];
  phys_flux(K, EK, d, FK);
  double rK = K[0], uK = K[1 + d], pK = K[4];
  double fac = rK * (SK - uK) / (SK - Ss);
  double Es = EK + (Ss - uK) * (Ss + pK / (rK * (SK - uK)));
  double Ws[5], WK[5];
  Ws[0] = fac;
  Ws[1] = fac * K[1];
  Ws[2] = fac * K[2];
  Ws[3] = fac * K[3];
  Ws[1 + d] = fac * Ss;
  Ws[4] = fac * Es;
  WK[0] = rK;
  WK[1] = rK * K[1];
  WK[2] = rK * K[2];
  WK[3] = rK * K[3];
  WK[4] = rK * EK;
  for (int v = 0; v < 5; ++v) F[v] = FK[v] + SK * (Ws[v] - WK[v]);
  return OR_OK;
}

/* Local Lax-Friedrichs flux (App. C.1, Eq. Lax-Friedrichs):
 * Phi = (F(W_L).n + F(W_R).n)/2 - lambda_max (W_R - W_L)/2 with
 * lambda_max = max(|u_L| + c_L, |u_R| + c_R), u the normal velocities. Inputs
 * are primitive states; one EOS for the whole face (Reading R15). */
static int llf(const or_eos_t* q, const double Lp[5], const double Rp[5], int d, double F[5]) {
  double c2L, c2R, eL, eR;
  int st = eos_c2(q, Lp[0], Lp[4], &c2L);
  if (!st) st = eos_c2(q, Rp[0], Rp[4], &c2R);
  if (!st) st = eos_e(q, Lp[0], Lp[4], &eL);
  if (!st) st = eos_e(q, Rp[0], Rp[4], &eR);
  if (st) return st;
  double EL = eL + 0.5 * ((Lp[1] * Lp[1] + Lp[2] * Lp[2]) + Lp[3] * Lp[3]);
  double ER = eR + 0.5 * ((Rp[1] * Rp[1] + Rp[2] * Rp[2]) + Rp[3] * Rp[3]);
  double lam = fmax(fabs(Lp[1 + d]) + sqrt(c2L), fabs(Rp[1 + d]) + sqrt(c2R));
  double FL[5], FR[5], WL[5], WR[5];
  phys_flux(Lp, EL, d, FL);
  phys_flux(Rp, ER, d, FR);
  WL[0] = Lp[0]; WL[1] = Lp[0] * Lp[1]; WL[2] = Lp[0] * Lp[2]; WL[3] = Lp[0] * Lp[3]; WL[4] = Lp[0] * EL;
  WR[0] = Rp[0]; WR[1] = Rp[0] * Rp[1]; WR[2] = Rp[0] * Rp[2]; WR[3] = Rp[0] * Rp[3]; WR[4] = Rp[0] * ER;
  for (int v = 0; v < 5; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (WR[v] - WL[v]);
  return OR_OK;
}

/* The numerical flux function Phi selected for the grid. */
static int num_flux(const or_grid_t* g, const or_eos_t* q, const double Lp[5], const double Rp[5], int d, double F[5]) {
  return g->flux == FLUX_LLF ? llf(q, Lp, Rp, d, F) : hllc(q, Lp, Rp, d, F);
}

/* ------------------------------------------------------------------ */
/* MUSCL reconstruction with the modified van Albada limiter, App. D    */
/* ------------------------------------------------------------------ */

/* Limited slope sigma = phi(theta) b with theta = a/b, uniform grid (A = B = 1),
 * k = 2: phi = (theta^2 + theta)/(theta^2 + 1) for theta >= 0 and 0 for theta < 0
 * (Reading R9, the modified limiter with its test read on theta). Written as
 * sigma = a b (a + b)/(a^2 + b^2) when a b > 0 (Reading R10: no division by b). */
static double va_slope(double a, double b) {
  if (!(a * b > 0.0)) return 0.0;
  return a * b * (a + b) / (a * a + b * b);
}

/* Monotonized central limiter (App. D, Eq. theta) on the uniform grid
 * (A = B = 1): phi(theta) = max(0, min(alpha theta, (theta + 1)/2, alpha)) and
 * sigma = phi(theta) b with theta = a/b. Reading R34: written without the
 * division, multiplying through by b (the inequalities turn for b < 0), and
 * sigma = 0 for b = 0 (phi(+-inf) b = 0). */
static double mc_slope(double a, double b, double alpha) {
  if (b > 0.0) return fmax(0.0, fmin(fmin(alpha * a, 0.5 * (a + b)), alpha * b));
  if (b < 0.0) return fmin(0.0, fmax(fmax(alpha * a, 0.5 * (a + b)), alpha * b));
  return 0.0;
}

static double limited_slope(const or_grid_t* g, double a, double b) {
  return g->limiter == LIM_MC ? mc_slope(a, b, g->mc_alpha) : va_slope(a, b);
}

/* ------------------------------------------------------------------ */
/* Grid helpers                                                          */
/* ------------------------------------------------------------------ */

/* Boundary conditions applied at every load (Reading R20/R26): a transmissive
 * side clamps the index (zero gradient), a periodic side wraps it, a symmetry
 * side mirrors it (the velocity component normal to the side is negated by
 * prim_at). */
static inline int map_index(int i, int n, int bclo, int bchi) {
  if (i < 0) return bclo == BC_PERIODIC ? ((i % n) + n) % n : (bclo == BC_SYMMETRY ? -1 - i : 0);
  if (i >= n) return bchi == BC_PERIODIC ? i % n : (bchi == BC_SYMMETRY ? 2 * n - 1 - i : n - 1);
  return i;
}

static inline long cell_index(const or_grid_t* g, int i, int j, int k) {
  i = map_index(i, g->n[0], g->bc[0], g->bc[1]);
  j = map_index(j, g->n[1], g->bc[2], g->bc[3]);
  k = map_index(k, g->n[2], g->bc[4], g->bc[5]);
  return ((long)k * g->n[1] + j) * g->n[0] + i;
}

static inline long ncells(const or_grid_t* g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static const int DIRV[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

/* Primitive state at the unmapped position (i,j,k): the mapped cell's, with the
 * velocity component normal to every symmetry side it was mirrored across
 * negated. */
static void prim_at(const or_grid_t* g, const double* P, int i, int j, int k, double out[5]) {
  long N = ncells(g), c = cell_index(g, i, j, k);
  for (int v = 0; v < 5; ++v) out[v] = P[v * N + c];
  const int x[3] = {i, j, k};
  for (int a = 0; a < 3; ++a)
    if ((x[a] < 0 && g->bc[2 * a] == BC_SYMMETRY) || (x[a] >= g->n[a] && g->bc[2 * a + 1] == BC_SYMMETRY))
      out[1 + a] = -out[1 + a];
}

static void record_error(int st, long cell, int* err, long* err_cell) {
#ifdef _OPENMP
#pragma omp critical(or_err)
#endif
  {
    if (*err == OR_OK || cell < *err_cell) {
      *err = st;
      *err_cell = cell;
    }
  }
}

/* Conservative -> primitive: u = (rho u)/rho, e = (rho E - rho|V|^2/2)/rho, p = p(rho, e). */
static int cons_to_prim(const or_eos_t* q, const double W[5], double P[5]) {
  double rho = W[0];
  if (!(rho > 0.0)) return OR_ENONPHYS;
  double u = W[1] / rho, v = W[2] / rho, w = W[3] / rho;
  double ke = 0.5 * ((W[1] * u + W[2] * v) + W[3] * w);
  double e = (W[4] - ke) / rho;
  double p;
  int st = eos_p(q, rho, e, &p);
  if (st) return st;
  double c2;
  st = eos_c2(q, rho, p, &c2);
  if (st) return st;
  P[0] = rho; P[1] = u; P[2] = v; P[3] = w; P[4] = p;
  return OR_OK;
}

static int prim_to_cons(const or_eos_t* q, const double P[5], double W[5]) {
  double e;
  int st = eos_e(q, P[0], P[4], &e);
  if (st) return st;
  W[0] = P[0];
  W[1] = P[0] * P[1];
  W[2] = P[0] * P[2];
  W[3] = P[0] * P[3];
  W[4] = P[0] * e + 0.5 * P[0] * ((P[1] * P[1] + P[2] * P[2]) + P[3] * P[3]);
  return OR_OK;
}

static int state_valid(const or_eos_t* q, const double Q[5]) {
  double c2;
  if (!(Q[0] > 0.0)) return 0;
  return eos_c2(q, Q[0], Q[4], &c2) == OR_OK;
}

/* Primitive states of all cells and material ids (ids from the sign of phi). */
static int all_prims(const or_grid_t* g, const double* W, const unsigned char* id, double* P, long* err_cell) {
  long N = ncells(g);
  int err = OR_OK;
  long ec = -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (long c = 0; c < N; ++c) {
    double w[5], p[5];
    for (int v = 0; v < 5; ++v) w[v] = W[v * N + c];
    int st = cons_to_prim(&g->eos[id[c]], w, p);
    if (st) {
      record_error(st, c, &err, &ec);
      for (int v = 0; v < 5; ++v) p[v] = NAN;
    }
    for (int v = 0; v < 5; ++v) P[v * N + c] = p[v];
  }
  if (err_cell) *err_cell = ec;
  return err;
}

/* Face states of the cell at (unmapped) position (i,j,k) in direction d:
 * Qm on its minus face, Qp on its plus face, q +- sigma/2 per primitive.
 * Reading R11: sigma = 0 when a stencil neighbour has another material.
 * Reading R12: sigma = 0 for all variables of this direction when a face state
 * is not admissible (rho <= 0 or c^2 <= 0). */
static void face_states(const or_grid_t* g, const double* P, const unsigned char* id, int i, int j, int k, int d,
                        double Qm[5], double Qp[5]) {
  long c = cell_index(g, i, j, k);
  long cm = cell_index(g, i - DIRV[d][0], j - DIRV[d][1], k - DIRV[d][2]);
  long cp = cell_index(g, i + DIRV[d][0], j + DIRV[d][1], k + DIRV[d][2]);
  int m = id[c];
  double Q[5], Qlo[5], Qhi[5];
  prim_at(g, P, i, j, k, Q);
  for (int v = 0; v < 5; ++v) Qm[v] = Qp[v] = Q[v];
  if (id[cm] != m || id[cp] != m) return;
  prim_at(g, P, i - DIRV[d][0], j - DIRV[d][1], k - DIRV[d][2], Qlo);
  prim_at(g, P, i + DIRV[d][0], j + DIRV[d][1], k + DIRV[d][2], Qhi);
  double tm[5], tp[5];
  for (int v = 0; v < 5; ++v) {
    double a = Q[v] - Qlo[v];
    double b = Qhi[v] - Q[v];
    double s = limited_slope(g, a, b);
    tm[v] = Q[v] - 0.5 * s;
    tp[v] = Q[v] + 0.5 * s;
  }
  if (!state_valid(&g->eos[m], tm) || !state_valid(&g->eos[m], tp)) return;
  for (int v = 0; v < 5; ++v) { Qm[v] = tm[v]; Qp[v] = tp[v]; }
}

/* Flux through the face between cell a at (i,j,k) and cell b = a + e_d, as seen
 * by cell a (side 0) or by cell b (side 1), Sec. 4.2. Same material: the MUSCL
 * flux Phi(W_ab, W_ba) with the grid's flux function (HLLC by default). Different materials (FIVER): the 1D
 * two-material Riemann problem of the normal projections gives W*_ab, W*_ba
 * (tangential velocity of each side's own face state, Reading R8), and
 * F_ab = Phi(W_ab, W*_ab; EOS_a), F_ba = Phi(W*_ba, W_ba; EOS_b) (Reading R16:
 * the left argument of Phi is always on the minus side of the face). */
static int face_flux(const or_grid_t* g, const double* P, const unsigned char* id, int i, int j, int k, int d,
                     int side, double F[5], int* iters) {
  int bi = i + DIRV[d][0], bj = j + DIRV[d][1], bk = k + DIRV[d][2];
  double Qa_m[5], Qa[5], Qb[5], Qb_p[5];
  face_states(g, P, id, i, j, k, d, Qa_m, Qa);
  face_states(g, P, id, bi, bj, bk, d, Qb, Qb_p);
  int ma = id[cell_index(g, i, j, k)], mb = id[cell_index(g, bi, bj, bk)];
  if (iters) *iters = 0;
  if (ma == mb) return num_flux(g, &g->eos[ma], Qa, Qb, d, F);
  double wa[3] = {Qa[0], Qa[1 + d], Qa[4]};
  double wb[3] = {Qb[0], Qb[1 + d], Qb[4]};
  double rs[4];
  int st = riemann(&g->eos[ma], wa, &g->eos[mb], wb, rs, iters);
  if (st) return st;
  double S[5];
  if (side == 0) {
    for (int v = 0; v < 5; ++v) S[v] = Qa[v];
    S[0] = rs[2];
    S[1 + d] = rs[1];
    S[4] = rs[0];
    return num_flux(g, &g->eos[ma], Qa, S, d, F);
  }
  for (int v = 0; v < 5; ++v) S[v] = Qb[v];
  S[0] = rs[3];
  S[1 + d] = rs[1];
  S[4] = rs[0];
  return num_flux(g, &g->eos[mb], S, Qb, d, F);
}

/* Narrow-band level set (Sec. 4.4: the level-set equation solved in a band
 * around the zero level set; Reading R38, the local level set of Peng et al.,
 * J. Comput. Phys. 155, 1999): the advection velocity is scaled by the cutoff
 * c(phi) = 1 for |phi| <= beta, (|phi| - gamma)^2 (2|phi| + gamma - 3 beta) /
 * (gamma - beta)^3 for beta < |phi| < gamma, 0 beyond, with beta and gamma the
 * tube radii (in cells times h), phi the cell's value in the stage; at the end
 * of the step (after the Runge-Kutta update and the scheduled
 * reinitialisation) phi is clipped to [-gamma, gamma], so that the level set
 * beyond the tube is a plateau at +-gamma that the tube's reinitialisation
 * pulls back to distances as the interface approaches. gamma = 0 is the full
 * domain. A reinitialisation restricted to |phi| < gamma would freeze the
 * plateau cells and, with the zero velocity at gamma, hold the tube's outer
 * edge in place (a sphere carried seven cells lagged a cell behind). */
static double band_cutoff(const or_grid_t* g, double phi) {
  double beta = g->band_beta * g->h, gamma = g->band_gamma * g->h, a = fabs(phi);
  if (a <= beta) return 1.0;
  if (a >= gamma) return 0.0;
  double d = gamma - beta;
  return (a - gamma) * (a - gamma) * (2.0 * a + gamma - 3.0 * beta) / (d * d * d);
}

static void band_clip(const or_grid_t* g, double* phi) {
  if (!(g->band_gamma > 0.0)) return;
  long N = ncells(g);
  double gamma = g->band_gamma * g->h;
  for (long c = 0; c < N; ++c) phi[c] = fmax(-gamma, fmin(gamma, phi[c]));
}

/* Third-order upwind-biased derivative of phi along d at cell c (Sec. 4.4,
 * Reading R18): for velocity >= 0, (2 phi_{+1} + 3 phi_0 - 6 phi_{-1} + phi_{-2})/(6h);
 * otherwise (-phi_{+2} + 6 phi_{+1} - 3 phi_0 - 2 phi_{-1})/(6h). */
static double ls_derivative(const or_grid_t* g, const double* phi, int i, int j, int k, int d, double vel) {
  int di = DIRV[d][0], dj = DIRV[d][1], dk = DIRV[d][2];
  double pm2 = phi[cell_index(g, i - 2 * di, j - 2 * dj, k - 2 * dk)];
  double pm1 = phi[cell_index(g, i - di, j - dj, k - dk)];
  double p0 = phi[cell_index(g, i, j, k)];
  double pp1 = phi[cell_index(g, i + di, j + dj, k + dk)];
  double pp2 = phi[cell_index(g, i + 2 * di, j + 2 * dj, k + 2 * dk)];
  if (vel >= 0.0) return (2.0 * pp1 + 3.0 * p0 - 6.0 * pm1 + pm2) / (6.0 * g->h);
  return (-pp2 + 6.0 * pp1 - 3.0 * p0 - 2.0 * pm1) / (6.0 * g->h);
}

/* Residual of one Runge-Kutta stage (Sec. 4.2, Eq. NS_discretized with G = S = 0):
 * R_i = -(1/|C_i|) sum_j F_ij, on the uniform grid
 * R = ((F_x- - F_x+)/h + (F_y- - F_y+)/h) + (F_z- - F_z+)/h in this association
 * (Reading R21 of the summation order), and the level-set residual
 * L = -((u phi_x + v phi_y) + w phi_z) (Sec. 3.5.1, Eq. levelset). Material ids
 * are those of the start of the step (Reading R19). */
static int stage_residual(const or_grid_t* g, const double* W, const double* phi, const unsigned char* id,
                          double* P, double* R, double* Lphi, or_stats_t* stats) {
  long N = ncells(g);
  long ec = -1;
  int err = all_prims(g, W, id, P, &ec);
  if (err) {
    if (stats) stats->err_cell = ec;
    return err;
  }
  long nif = 0, itmax = 0;
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : nif) reduction(max : itmax) collapse(2)
#endif
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        double acc[5] = {0, 0, 0, 0, 0};
        int st = OR_OK;
        for (int d = 0; d < 3 && !st; ++d) {
          double Fm[5], Fp[5];
          int itm = 0, itp = 0;
          st = face_flux(g, P, id, i - DIRV[d][0], j - DIRV[d][1], k - DIRV[d][2], d, 1, Fm, &itm);
          if (!st) st = face_flux(g, P, id, i, j, k, d, 0, Fp, &itp);
          if (st) break;
          if (id[cell_index(g, i + DIRV[d][0], j + DIRV[d][1], k + DIRV[d][2])] != id[c]) nif += 1;
          if (itm > itmax) itmax = itm;
          if (itp > itmax) itmax = itp;
          for (int v = 0; v < 5; ++v) acc[v] = acc[v] + (Fm[v] - Fp[v]) / g->h;
        }
        if (st) {
          record_error(st, c, &err, &ec);
          continue;
        }
        if (g->geom != GEOM_CARTESIAN) {
          /* Sec. 3.4: S = -(alpha/r) u_r (rho, rho u, rho v, rho w, rho E + p), alpha = 1
           * (cylindrical) or 2 (spherical); Reading R37: evaluated at the cell centre
           * r = x0 + (i + 1/2) h from the stage state, added after the flux sum */
          double r = g->x0 + (i + 0.5) * g->h;
          double a = (g->geom == GEOM_SPHERICAL ? 2.0 : 1.0) / r * P[1 * N + c];
          for (int v = 0; v < 4; ++v) acc[v] = acc[v] - a * W[v * N + c];
          acc[4] = acc[4] - a * (W[4 * N + c] + P[4 * N + c]);
        }
        for (int v = 0; v < 5; ++v) R[v * N + c] = acc[v];
        double u = P[1 * N + c], v = P[2 * N + c], w = P[3 * N + c];
        double Dx = ls_derivative(g, phi, i, j, k, 0, u);
        double Dy = ls_derivative(g, phi, i, j, k, 1, v);
        double Dz = ls_derivative(g, phi, i, j, k, 2, w);
        Lphi[c] = -((u * Dx + v * Dy) + w * Dz);
        if (g->band_gamma > 0.0) Lphi[c] = band_cutoff(g, phi[c]) * Lphi[c];
      }
  if (stats) {
    stats->interface_faces = nif;
    if (itmax > stats->newton_max) stats->newton_max = itmax;
    if (err) stats->err_cell = ec;
  }
  return err;
}

/* Time step from a CFL number (Sec. 4.3). Reading R21: for the unsplit 3D
 * scheme the CFL condition is applied to the sum over the directions with more
 * than one cell, dt = CFL h / max_i sum_d (|V_d| + c). */
static int time_step(const or_grid_t* g, const double* W, const unsigned char* id, double* P, double* dt, long* err_cell) {
  long N = ncells(g);
  int st = all_prims(g, W, id, P, err_cell);
  if (st) return st;
  double lmax = 0.0;
  int err = OR_OK;
  long ec = -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(max : lmax)
#endif
  for (long c = 0; c < N; ++c) {
    double c2;
    int s2 = eos_c2(&g->eos[id[c]], P[c], P[4 * N + c], &c2);
    if (s2) {
      record_error(s2, c, &err, &ec);
      continue;
    }
    double cs = sqrt(c2), lam = 0.0;
    for (int d = 0; d < 3; ++d)
      if (g->n[d] > 1) lam = lam + (fabs(P[(1 + d) * N + c]) + cs);
    if (lam > lmax) lmax = lam;
  }
  if (err) {
    if (err_cell) *err_cell = ec;
    return err;
  }
  if (!(lmax > 0.0) || !isfinite(lmax)) return OR_ENONPHYS;
  *dt = g->cfl * g->h / lmax;
  return OR_OK;
}

/* Reinitialisation (Sec. 3.5.1, Eq. reinit; Sec. 4.4): N pseudo-time steps of
 * phi^{k+1} = phi^k - dtau S(phi0) (G(phi^k) - 1) with the upwind Godunov
 * gradient norm G, S(phi0) = phi0/sqrt(phi0^2 + eps^2), eps = h, dtau = h/2
 * (Reading R24), cells with a face neighbour of the other sign held fixed
 * (Reading R25, the "fixed first layer" option). Jacobi sweeps. */
static void reinit(const or_grid_t* g, double* phi, int iters, double* phi0, double* tmp) {
  long N = ncells(g);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const double h = g->h, dtau = 0.5 * g->h;
  memcpy(phi0, phi, sizeof(double) * N);
  double* cur = phi;
  double* nxt = tmp;
  for (int it = 0; it < iters; ++it) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) collapse(2)
#endif
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          long c = ((long)k * ny + j) * nx + i;
          int s0 = phi0[c] < 0.0;
          int first = 0;
          for (int d = 0; d < 3; ++d) {
            long cm = cell_index(g, i - DIRV[d][0], j - DIRV[d][1], k - DIRV[d][2]);
            long cp = cell_index(g, i + DIRV[d][0], j + DIRV[d][1], k + DIRV[d][2]);
            if ((phi0[cm] < 0.0) != s0 || (phi0[cp] < 0.0) != s0) first = 1;
          }
          if (first) {
            nxt[c] = cur[c];
            continue;
          }
          double G2[3];
          for (int d = 0; d < 3; ++d) {
            long cm = cell_index(g, i - DIRV[d][0], j - DIRV[d][1], k - DIRV[d][2]);
            long cp = cell_index(g, i + DIRV[d][0], j + DIRV[d][1], k + DIRV[d][2]);
            double a = (cur[c] - cur[cm]) / h;
            double b = (cur[cp] - cur[c]) / h;
            double x, y;
            if (phi0[c] >= 0.0) {
              x = fmax(a, 0.0);
              y = fmin(b, 0.0);
            } else {
              x = fmin(a, 0.0);
              y = fmax(b, 0.0);
            }
            G2[d] = fmax(x * x, y * y);
          }
          double G = sqrt((G2[0] + G2[1]) + G2[2]);
          double S = phi0[c] / sqrt(phi0[c] * phi0[c] + h * h);
          nxt[c] = cur[c] - dtau * S * (G - 1.0);
        }
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != phi) memcpy(phi, cur, sizeof(double) * N);
}

/* Phase update, Sec. 2.3 step (6). Reading R17: a cell whose material changed
 * takes the arithmetic mean of the primitive states of its face neighbours
 * (order x-, x+, y-, y+, z-, z+) that were and still are of its new material,
 * converted with the new EOS; if there is none, the 26-neighbourhood (z, y, x
 * loops from -1 to 1) is used; if there is still none (a material fragment
 * smaller than a cell, e.g. a level-set undershoot), the cell keeps its old
 * material and state and its level set takes the old material's sign:
 * phi = |phi| for material 0, phi = -max(|phi|, 1e-12 h) for material 1. */
static int phase_fix(const or_grid_t* g, double* W, double* phi, const unsigned char* id_old,
                     const unsigned char* id_new, double* P, long* nflip, long* err_cell) {
  long N = ncells(g);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  /* primitive states of the cells that keep their material */
  int err = OR_OK;
  long ec = -1, nf = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (long c = 0; c < N; ++c) {
    double w[5], p[5];
    for (int v = 0; v < 5; ++v) w[v] = W[v * N + c];
    if (id_old[c] == id_new[c] && cons_to_prim(&g->eos[id_new[c]], w, p) == OR_OK) {
      for (int v = 0; v < 5; ++v) P[v * N + c] = p[v];
    } else {
      for (int v = 0; v < 5; ++v) P[v * N + c] = NAN;
    }
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(static) collapse(2) reduction(+ : nf)
#endif
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        if (id_old[c] == id_new[c]) continue;
        nf += 1;
        int m = id_new[c];
        double sum[5] = {0, 0, 0, 0, 0};
        int cnt = 0;
        for (int d = 0; d < 3; ++d)
          for (int sgn = -1; sgn <= 1; sgn += 2) {
            long nb = cell_index(g, i + sgn * DIRV[d][0], j + sgn * DIRV[d][1], k + sgn * DIRV[d][2]);
            if (id_old[nb] == m && id_new[nb] == m) {
              double q[5];
              prim_at(g, P, i + sgn * DIRV[d][0], j + sgn * DIRV[d][1], k + sgn * DIRV[d][2], q);
              for (int v = 0; v < 5; ++v) sum[v] = sum[v] + q[v];
              cnt += 1;
            }
          }
        if (cnt == 0) {
          for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
              for (int di = -1; di <= 1; ++di) {
                if (!di && !dj && !dk) continue;
                long nb = cell_index(g, i + di, j + dj, k + dk);
                if (id_old[nb] == m && id_new[nb] == m) {
                  double q[5];
                  prim_at(g, P, i + di, j + dj, k + dk, q);
                  for (int v = 0; v < 5; ++v) sum[v] = sum[v] + q[v];
                  cnt += 1;
                }
              }
        }
        if (cnt == 0) {
          phi[c] = id_old[c] ? -fmax(fabs(phi[c]), 1e-12 * g->h) : fabs(phi[c]);
          continue;
        }
        double pr[5], w[5];
        for (int v = 0; v < 5; ++v) pr[v] = sum[v] / cnt;
        int st = prim_to_cons(&g->eos[m], pr, w);
        if (st) {
          record_error(st, c, &err, &ec);
          continue;
        }
        for (int v = 0; v < 5; ++v) W[v * N + c] = w[v];
      }
  if (nflip) *nflip = nf;
  if (err && err_cell) *err_cell = ec;
  return err;
}

/* ------------------------------------------------------------------ */
/* One time step, Sec. 2.3 steps (1)-(6) with the second-order TVD      */
/* Runge-Kutta schemes of Sec. 4.3 (TVD RK2 by default, TVD RK3, forward */
/* Euler); RK2: W1 = W + dt R(W), W' = (W + (W1 + dt R(W1)))/2, and the */
/* same for phi.                                                         */
/* ------------------------------------------------------------------ */

typedef struct {
  double *W1, *phi1, *P, *R, *L, *tmp0, *tmp1;
  unsigned char *id, *id2;
} work_t;

static void work_free(work_t* w) {
  free(w->W1); free(w->phi1); free(w->P); free(w->R); free(w->L); free(w->tmp0); free(w->tmp1);
  free(w->id); free(w->id2);
}

static int work_alloc(work_t* w, long N) {
  memset(w, 0, sizeof(*w));
  w->W1 = malloc(sizeof(double) * 5 * N);
  w->phi1 = malloc(sizeof(double) * N);
  w->P = malloc(sizeof(double) * 5 * N);
  w->R = malloc(sizeof(double) * 5 * N);
  w->L = malloc(sizeof(double) * N);
  w->tmp0 = malloc(sizeof(double) * N);
  w->tmp1 = malloc(sizeof(double) * N);
  w->id = malloc(N);
  w->id2 = malloc(N);
  if (!w->W1 || !w->phi1 || !w->P || !w->R || !w->L || !w->tmp0 || !w->tmp1 || !w->id || !w->id2) {
    work_free(w);
    return OR_ENOMEM;
  }
  return OR_OK;
}

static int step_one(const or_grid_t* g, double* W, double* phi, long step_index, work_t* wk, or_stats_t* stats) {
  long N = ncells(g);
  for (long c = 0; c < N; ++c) wk->id[c] = phi[c] < 0.0;
  double dt;
  long ec = -1;
  int st = time_step(g, W, wk->id, wk->P, &dt, &ec);
  if (st) {
    stats->err_cell = ec;
    return st;
  }
  if (g->dt_fixed > 0.0) dt = g->dt_fixed; /* Sec. 4.3: a constant time step instead of the CFL rule */
  stats->dt = dt;
  /* stage 1: W1 = W + dt R(W), the same for phi */
  st = stage_residual(g, W, phi, wk->id, wk->P, wk->R, wk->L, stats);
  if (st) return st;
  long nif1 = stats->interface_faces;
  if (g->rk == 1) { /* forward Euler (Sec. 4.3) */
    for (long x = 0; x < 5 * N; ++x) W[x] = W[x] + dt * wk->R[x];
    for (long c = 0; c < N; ++c) phi[c] = phi[c] + dt * wk->L[c];
  } else {
    for (long x = 0; x < 5 * N; ++x) wk->W1[x] = W[x] + dt * wk->R[x];
    for (long c = 0; c < N; ++c) wk->phi1[c] = phi[c] + dt * wk->L[c];
    /* stage 2, material ids frozen */
    st = stage_residual(g, wk->W1, wk->phi1, wk->id, wk->P, wk->R, wk->L, stats);
    if (st) return st;
    if (g->rk == 3) {
      /* TVD RK3 (Sec. 4.3): W2 = 3/4 W + 1/4 W1 + 1/4 dt R(W1) (into W1), then
       * W' = 1/3 W + 2/3 W2 + 2/3 dt R(W2), each sum taken left to right */
      for (long x = 0; x < 5 * N; ++x) wk->W1[x] = (0.75 * W[x] + 0.25 * wk->W1[x]) + 0.25 * dt * wk->R[x];
      for (long c = 0; c < N; ++c) wk->phi1[c] = (0.75 * phi[c] + 0.25 * wk->phi1[c]) + 0.25 * dt * wk->L[c];
      st = stage_residual(g, wk->W1, wk->phi1, wk->id, wk->P, wk->R, wk->L, stats);
      if (st) return st;
      for (long x = 0; x < 5 * N; ++x)
        W[x] = (W[x] / 3.0 + 2.0 / 3.0 * wk->W1[x]) + 2.0 / 3.0 * dt * wk->R[x];
      for (long c = 0; c < N; ++c) phi[c] = (phi[c] / 3.0 + 2.0 / 3.0 * wk->phi1[c]) + 2.0 / 3.0 * dt * wk->L[c];
    } else {
      /* TVD RK2: W' = (W + (W1 + dt R(W1)))/2 */
      for (long x = 0; x < 5 * N; ++x) W[x] = 0.5 * (W[x] + (wk->W1[x] + dt * wk->R[x]));
      for (long c = 0; c < N; ++c) phi[c] = 0.5 * (phi[c] + (wk->phi1[c] + dt * wk->L[c]));
    }
  }
  stats->interface_faces = nif1;
  /* (5) reinitialisation when scheduled: after steps reinit_every, 2 reinit_every, ... */
  if (g->reinit_every > 0 && g->reinit_iters > 0 && (step_index + 1) % g->reinit_every == 0)
    reinit(g, phi, g->reinit_iters, wk->tmp0, wk->tmp1);
  band_clip(g, phi); /* narrow band (Reading R38) */
  /* (6) phase update */
  for (long c = 0; c < N; ++c) wk->id2[c] = phi[c] < 0.0;
  long nf = 0;
  st = phase_fix(g, W, phi, wk->id, wk->id2, wk->P, &nf, &ec);
  stats->flipped = nf;
  if (st) stats->err_cell = ec;
  return st;
}

/* ------------------------------------------------------------------ */
/* Exact solution sampler for two stiffened gases (closed form)          */
/* ------------------------------------------------------------------ */

/* State at x/t = xi of the exact solution whose star values are given.
 * Rarefaction fans use the SG isentrope in p + p_c and c^2 = gamma (p + p_c)/rho. */
static void sample_sg(double gL, double pcL, const double wL[3], double gR, double pcR, const double wR[3],
                      const double star[4], double xi, double out[3]) {
  double ps = star[0], us = star[1];
  if (xi <= us) {
    double g = gL, pc = pcL, rho = wL[0], u = wL[1], p = wL[2];
    double c = sqrt(g * (p + pc) / rho), pb = p + pc, pbs = ps + pc;
    if (ps > p) {
      double S = u - c * sqrt((g + 1.0) / (2.0 * g) * pbs / pb + (g - 1.0) / (2.0 * g));
      if (xi <= S) { out[0] = rho; out[1] = u; out[2] = p; }
      else { out[0] = star[2]; out[1] = us; out[2] = ps; }
    } else {
      double cs = c * pow(pbs / pb, (g - 1.0) / (2.0 * g));
      double head = u - c, tail = us - cs;
      if (xi <= head) { out[0] = rho; out[1] = u; out[2] = p; }
      else if (xi >= tail) { out[0] = star[2]; out[1] = us; out[2] = ps; }
      else {
        double uf = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * u + xi);
        double cf = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * (u - xi));
        out[0] = rho * pow(cf / c, 2.0 / (g - 1.0));
        out[1] = uf;
        out[2] = pb * pow(cf / c, 2.0 * g / (g - 1.0)) - pc;
      }
    }
  } else {
    double g = gR, pc = pcR, rho = wR[0], u = wR[1], p = wR[2];
    double c = sqrt(g * (p + pc) / rho), pb = p + pc, pbs = ps + pc;
    if (ps > p) {
      double S = u + c * sqrt((g + 1.0) / (2.0 * g) * pbs / pb + (g - 1.0) / (2.0 * g));
      if (xi >= S) { out[0] = rho; out[1] = u; out[2] = p; }
      else { out[0] = star[3]; out[1] = us; out[2] = ps; }
    } else {
      double cs = c * pow(pbs / pb, (g - 1.0) / (2.0 * g));
      double head = u + c, tail = us + cs;
      if (xi >= head) { out[0] = rho; out[1] = u; out[2] = p; }
      else if (xi <= tail) { out[0] = star[3]; out[1] = us; out[2] = ps; }
      else {
        double uf = 2.0 / (g + 1.0) * (-c + 0.5 * (g - 1.0) * u + xi);
        double cf = 2.0 / (g + 1.0) * (c - 0.5 * (g - 1.0) * (u - xi));
        out[0] = rho * pow(cf / c, 2.0 / (g - 1.0));
        out[1] = uf;
        out[2] = pb * pow(cf / c, 2.0 * g / (g - 1.0)) - pc;
      }
    }
  }
}

/* ------------------------------------------------------------------ */
/* Exported entry points (flat arguments for ctypes)                    */
/* ------------------------------------------------------------------ */

static void mk_eos(or_eos_t* q, int type, const double* prm) {
  q->type = type;
  for (int i = 0; i < 6; ++i) q->prm[i] = prm[i];
}

/* ip = {nx, ny, nz, bc[6], reinit_every, reinit_iters, eos_type0, eos_type1, nthreads,
 *       rk, limiter, flux, geom}
 * dp = {h, cfl, eos_prm0[6], eos_prm1[6], mc_alpha, dt_fixed, x0} */
static int mk_grid(or_grid_t* g, const int* ip, const double* dp) {
  for (int a = 0; a < 3; ++a) g->n[a] = ip[a];
  for (int s = 0; s < 6; ++s) g->bc[s] = ip[3 + s];
  g->reinit_every = ip[9];
  g->reinit_iters = ip[10];
  mk_eos(&g->eos[0], ip[11], dp + 2);
  mk_eos(&g->eos[1], ip[12], dp + 8);
  g->h = dp[0];
  g->cfl = dp[1];
  g->rk = ip[14];
  g->limiter = ip[15];
  g->flux = ip[16];
  g->mc_alpha = dp[14];
  g->dt_fixed = dp[15];
  g->geom = ip[17];
  g->x0 = dp[16];
  g->band_beta = dp[17];
  g->band_gamma = dp[18];
#ifdef _OPENMP
  if (ip[13] > 0) omp_set_num_threads(ip[13]);
#endif
  for (int a = 0; a < 3; ++a) {
    if (g->n[a] < 1) return OR_EINVAL;
    if ((g->bc[2 * a] == BC_PERIODIC) != (g->bc[2 * a + 1] == BC_PERIODIC)) return OR_EINVAL;
    for (int sd = 0; sd < 2; ++sd) {
      int b = g->bc[2 * a + sd];
      if (b != BC_TRANSMISSIVE && b != BC_PERIODIC && b != BC_SYMMETRY) return OR_EINVAL;
      if (b == BC_SYMMETRY && g->n[a] < 2) return OR_EINVAL; /* a two-cell mirror needs two cells */
    }
  }
  if (g->geom != GEOM_CARTESIAN && g->geom != GEOM_CYLINDRICAL && g->geom != GEOM_SPHERICAL) return OR_EINVAL;
  if (g->geom != GEOM_CARTESIAN && (!(g->x0 >= 0.0) || g->n[1] != 1)) return OR_EINVAL;
  if (g->geom == GEOM_SPHERICAL && g->n[2] != 1) return OR_EINVAL;
  /* at least one axis with more than one cell: otherwise nothing moves and the time step is undefined */
  if (g->n[0] * g->n[1] * g->n[2] < 2) return OR_EINVAL;
  if (!(g->h > 0.0)) return OR_EINVAL;
  for (int m = 0; m < 2; ++m)
    if (g->eos[m].type != EOS_SG && g->eos[m].type != EOS_MG && g->eos[m].type != EOS_NASG &&
        g->eos[m].type != EOS_JWL)
      return OR_EINVAL;
  if (g->rk != 1 && g->rk != 2 && g->rk != 3) return OR_EINVAL;
  if (g->limiter != LIM_VA_MOD && g->limiter != LIM_MC) return OR_EINVAL;
  if (g->flux != FLUX_HLLC && g->flux != FLUX_LLF) return OR_EINVAL;
  if (g->limiter == LIM_MC && !(g->mc_alpha >= 0.0 && g->mc_alpha <= 2.0)) return OR_EINVAL;
  if (!(g->dt_fixed >= 0.0)) return OR_EINVAL;
  if (g->band_gamma > 0.0 && !(g->band_beta > 0.0 && g->band_beta < g->band_gamma)) return OR_EINVAL;
  return OR_OK;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int or_eos_pressure(int type, const double* prm, double rho, double e, double* p) {
  or_eos_t q; mk_eos(&q, type, prm); return eos_p(&q, rho, e, p);
}
int or_eos_energy(int type, const double* prm, double rho, double p, double* e) {
  or_eos_t q; mk_eos(&q, type, prm); return eos_e(&q, rho, p, e);
}
int or_eos_c2(int type, const double* prm, double rho, double p, double* c2) {
  or_eos_t q; mk_eos(&q, type, prm); return eos_c2(&q, rho, p, c2);
}

/* out = {f, df/dp, rho behind the wave} for the wave of one side at pressure p */
int or_wave_curve(int type, const double* prm, const double* w, double p, double* out) {
  or_eos_t q; mk_eos(&q, type, prm);
  side_t K;
  int st = make_side(&q, w, &K);
  if (st) return st;
  return wave(&q, &K, p, &out[0], &out[1], &out[2]);
}

int or_riemann(int typeL, const double* prmL, const double* wL, int typeR, const double* prmR, const double* wR,
               double* out, int* iters) {
  or_eos_t qL, qR; mk_eos(&qL, typeL, prmL); mk_eos(&qR, typeR, prmR);
  return riemann(&qL, wL, &qR, wR, out, iters);
}

/* batch of n problems, SoA inputs L[3n], R[3n], out[4n] */
int or_riemann_batch(int n, int typeL, const double* prmL, const double* L, int typeR, const double* prmR,
                     const double* R, double* out, int* iters, int* status) {
  or_eos_t qL, qR; mk_eos(&qL, typeL, prmL); mk_eos(&qR, typeR, prmR);
  int first = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (int i = 0; i < n; ++i) {
    double wl[3] = {L[i], L[n + i], L[2 * n + i]}, wr[3] = {R[i], R[n + i], R[2 * n + i]}, o[4];
    int it = 0;
    int st = riemann(&qL, wl, &qR, wr, o, &it);
    for (int v = 0; v < 4; ++v) out[v * n + i] = st ? NAN : o[v];
    if (iters) iters[i] = it;
    if (status) status[i] = st;
  }
  if (status)
    for (int i = 0; i < n; ++i)
      if (status[i]) { first = status[i]; break; }
  return first;
}

int or_hllc(int type, const double* prm, const double* qL, const double* qR, int d, double* F) {
  or_eos_t q; mk_eos(&q, type, prm);
  return hllc(&q, qL, qR, d, F);
}

double or_va_slope(double a, double b) { return va_slope(a, b); }

double or_band_cutoff(double beta, double gamma, double h, double phi) {
  or_grid_t g;
  memset(&g, 0, sizeof(g));
  g.band_beta = beta;
  g.band_gamma = gamma;
  g.h = h;
  return band_cutoff(&g, phi);
}

double or_mc_slope(double a, double b, double alpha) { return mc_slope(a, b, alpha); }

int or_llf(int type, const double* prm, const double* qL, const double* qR, int d, double* F) {
  or_eos_t q;
  mk_eos(&q, type, prm);
  return llf(&q, qL, qR, d, F);
}

/* Post-shock state of a shock moving in +x into the state w = (rho, u, p) at
 * pressure p1 behind it: out = {rho1, u1, shock speed}. The shocked state is
 * the star state of the right-facing wave: u1 = u + f(p1). */
int or_shock_state(int type, const double* prm, const double* w, double p1, double* out) {
  or_eos_t q; mk_eos(&q, type, prm);
  side_t K;
  int st = make_side(&q, w, &K);
  if (st) return st;
  if (!(p1 > K.p)) return OR_EINVAL;
  double f, df, rs;
  st = wave(&q, &K, p1, &f, &df, &rs);
  if (st) return st;
  out[0] = rs;
  out[1] = K.u + f;
  out[2] = (rs * out[1] - K.rho * K.u) / (rs - K.rho);
  return OR_OK;
}

/* prims (5N) and phi -> W (5N); the material of each cell from the sign of phi */
int or_prims_to_cons(const int* ip, const double* dp, const double* prims, const double* phi, double* W) {
  or_grid_t g;
  int st = mk_grid(&g, ip, dp);
  if (st) return st;
  long N = ncells(&g);
  for (long c = 0; c < N; ++c) {
    double p[5], w[5];
    for (int v = 0; v < 5; ++v) p[v] = prims[v * N + c];
    st = prim_to_cons(&g.eos[phi[c] < 0.0], p, w);
    if (st) return st;
    for (int v = 0; v < 5; ++v) W[v * N + c] = w[v];
  }
  return OR_OK;
}

int or_cons_to_prims(const int* ip, const double* dp, const double* W, const double* phi, double* prims) {
  or_grid_t g;
  int st = mk_grid(&g, ip, dp);
  if (st) return st;
  long N = ncells(&g);
  unsigned char* id = malloc(N);
  if (!id) return OR_ENOMEM;
  for (long c = 0; c < N; ++c) id[c] = phi[c] < 0.0;
  st = all_prims(&g, W, id, prims, NULL);
  free(id);
  return st;
}

int or_time_step(const int* ip, const double* dp, const double* W, const double* phi, double* dt) {
  or_grid_t g;
  int st = mk_grid(&g, ip, dp);
  if (st) return st;
  long N = ncells(&g);
  unsigned char* id = malloc(N);
  double* P = malloc(sizeof(double) * 5 * N);
  if (!id || !P) { free(id); free(P); return OR_ENOMEM; }
  for (long c = 0; c < N; ++c) id[c] = phi[c] < 0.0;
  st = time_step(&g, W, id, P, dt, NULL);
  free(id); free(P);
  return st;
}

/* One stage residual: R (5N), L (N); stats = {interface faces, newton max} */
int or_residual(const int* ip, const double* dp, const double* W, const double* phi, double* R, double* L, long* stats) {
  or_grid_t g;
  int st = mk_grid(&g, ip, dp);
  if (st) return st;
  long N = ncells(&g);
  unsigned char* id = malloc(N);
  double* P = malloc(sizeof(double) * 5 * N);
  if (!id || !P) { free(id); free(P); return OR_ENOMEM; }
  for (long c = 0; c < N; ++c) id[c] = phi[c] < 0.0;
  or_stats_t s = {0, 0, 0, 0, -1};
  st = stage_residual(&g, W, phi, id, P, R, L, &s);
  if (stats) { stats[0] = s.interface_faces; stats[1] = s.newton_max; stats[2] = s.err_cell; }
  free(id); free(P);
  return st;
}

/* nsteps time steps starting at step index step0; t advanced by the sum of dt.
 * stats = {last dt bits not used; interface faces, newton max, flipped total, err cell} */
int or_run(const int* ip, const double* dp, double* W, double* phi, long step0, int nsteps, double* t, long* stats,
           double* dts) {
  or_grid_t g;
  int st = mk_grid(&g, ip, dp);
  if (st) return st;
  long N = ncells(&g);
  work_t wk;
  st = work_alloc(&wk, N);
  if (st) return st;
  or_stats_t s = {0, 0, 0, 0, -1};
  long flipped = 0;
  for (int n = 0; n < nsteps; ++n) {
    st = step_one(&g, W, phi, step0 + n, &wk, &s);
    if (st) break;
    if (t) *t = *t + s.dt;
    if (dts) dts[n] = s.dt;
    flipped += s.flipped;
  }
  if (stats) { stats[0] = s.interface_faces; stats[1] = s.newton_max; stats[2] = flipped; stats[3] = s.err_cell; }
  work_free(&wk);
  return st;
}

/* The phase update alone (Sec. 2.3 step (6), Reading R17) on (W, phi) with the
 * material ids id_old of the start of the step; the new ids are sign(phi).
 * nflip: cells that changed material. */
int or_phase_fix(const int* ip, const double* dp, double* W, double* phi, const unsigned char* id_old, long* nflip) {
  or_grid_t g;
  int st = mk_grid(&g, ip, dp);
  if (st) return st;
  long N = ncells(&g);
  unsigned char* id_new = malloc(N);
  double* P = malloc(sizeof(double) * 5 * N);
  if (!id_new || !P) { free(id_new); free(P); return OR_ENOMEM; }
  for (long c = 0; c < N; ++c) id_new[c] = phi[c] < 0.0;
  long ec = -1;
  st = phase_fix(&g, W, phi, id_old, id_new, P, nflip, &ec);
  free(id_new); free(P);
  return st;
}

int or_reinit(const int* ip, const double* dp, double* phi, int iters) {
  or_grid_t g;
  int st = mk_grid(&g, ip, dp);
  if (st) return st;
  long N = ncells(&g);
  double* a = malloc(sizeof(double) * N);
  double* b = malloc(sizeof(double) * N);
  if (!a || !b) { free(a); free(b); return OR_ENOMEM; }
  reinit(&g, phi, iters, a, b);
  free(a); free(b);
  return OR_OK;
}

/* Exact solution of a two-stiffened-gas Riemann problem sampled at n points xi = x/t.
 * out = {rho[n], u[n], p[n]}, star = {p*, u*, rho*L, rho*R}. */
int or_exact_sample_sg(const double* prmL, const double* wL, const double* prmR, const double* wR, int n,
                       const double* xi, double* out, double* star) {
  or_eos_t qL, qR; mk_eos(&qL, EOS_SG, prmL); mk_eos(&qR, EOS_SG, prmR);
  double s[4];
  int it;
  int st = riemann(&qL, wL, &qR, wR, s, &it);
  if (st) return st;
  for (int i = 0; i < n; ++i) {
    double o[3];
    sample_sg(prmL[0], prmL[1], wL, prmR[0], prmR[1], wR, s, xi[i], o);
    out[i] = o[0];
    out[n + i] = o[1];
    out[2 * n + i] = o[2];
  }
  if (star) for (int v = 0; v < 4; ++v) star[v] = s[v];
  return OR_OK;
}
