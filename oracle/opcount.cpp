// Op-counting build of the oracle (TEST AND MEASUREMENT INFRASTRUCTURE ONLY, like
// the oracle itself): m2c_oracle.c compiled as C++ with its floating-point type
// replaced by a type that counts every FP64 addition or subtraction,
// multiplication, division and square root it performs (transcendental calls
// are counted apart). The oracle's arithmetic is unchanged; this file only
// supplies the type and a harness that calls the oracle's own functions once per
// face and once per cell, as one time step of the method needs them (the oracle
// itself, written for clarity, computes each face's flux twice). Build and use:
// oracle/count_flops.py. Nothing in the GPU solver includes or calls this.
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace opc {
struct Counts {
  unsigned long long add, mul, div, sqrt, special;
};
Counts g;
}  // namespace opc

struct cnt_t {
  double v;
  cnt_t() = default;
  cnt_t(double x) : v(x) {}
  operator double() const { return v; }
  cnt_t& operator+=(cnt_t o) { ++opc::g.add; v += o.v; return *this; }
  cnt_t& operator-=(cnt_t o) { ++opc::g.add; v -= o.v; return *this; }
  cnt_t& operator*=(cnt_t o) { ++opc::g.mul; v *= o.v; return *this; }
  cnt_t& operator/=(cnt_t o) { ++opc::g.div; v /= o.v; return *this; }
};
static inline cnt_t operator-(cnt_t a) { return cnt_t(-a.v); }
#define OPC_BIN(OP, FIELD)                                                                \
  static inline cnt_t operator OP(cnt_t a, cnt_t b) { ++opc::g.FIELD; return cnt_t(a.v OP b.v); } \
  static inline cnt_t operator OP(cnt_t a, double b) { ++opc::g.FIELD; return cnt_t(a.v OP b); }  \
  static inline cnt_t operator OP(double a, cnt_t b) { ++opc::g.FIELD; return cnt_t(a OP b.v); }  \
  static inline cnt_t operator OP(cnt_t a, int b) { ++opc::g.FIELD; return cnt_t(a.v OP b); }     \
  static inline cnt_t operator OP(int a, cnt_t b) { ++opc::g.FIELD; return cnt_t(a OP b.v); }     \
  static inline cnt_t operator OP(cnt_t a, long b) { ++opc::g.FIELD; return cnt_t(a.v OP b); }    \
  static inline cnt_t operator OP(long a, cnt_t b) { ++opc::g.FIELD; return cnt_t(a OP b.v); }
OPC_BIN(+, add)
OPC_BIN(-, add)
OPC_BIN(*, mul)
OPC_BIN(/, div)
#undef OPC_BIN
#define OPC_CMP(OP)                                                                   \
  static inline bool operator OP(cnt_t a, cnt_t b) { return a.v OP b.v; }            \
  static inline bool operator OP(cnt_t a, double b) { return a.v OP b; }             \
  static inline bool operator OP(double a, cnt_t b) { return a OP b.v; }             \
  static inline bool operator OP(cnt_t a, int b) { return a.v OP b; }                \
  static inline bool operator OP(int a, cnt_t b) { return a OP b.v; }
OPC_CMP(<)
OPC_CMP(>)
OPC_CMP(<=)
OPC_CMP(>=)
OPC_CMP(==)
OPC_CMP(!=)
#undef OPC_CMP
static inline cnt_t sqrt(cnt_t a) { ++opc::g.sqrt; return cnt_t(std::sqrt(a.v)); }
static inline cnt_t fabs(cnt_t a) { return cnt_t(std::fabs(a.v)); }
static inline cnt_t exp(cnt_t a) { ++opc::g.special; return cnt_t(std::exp(a.v)); }
static inline cnt_t log(cnt_t a) { ++opc::g.special; return cnt_t(std::log(a.v)); }
static inline cnt_t pow(cnt_t a, cnt_t b) { ++opc::g.special; return cnt_t(std::pow(a.v, b.v)); }
static inline cnt_t pow(cnt_t a, double b) { ++opc::g.special; return cnt_t(std::pow(a.v, b)); }
static inline cnt_t ceil(cnt_t a) { return cnt_t(std::ceil(a.v)); }
static inline cnt_t fmax(cnt_t a, cnt_t b) { return cnt_t(std::fmax(a.v, b.v)); }
static inline cnt_t fmax(cnt_t a, double b) { return cnt_t(std::fmax(a.v, b)); }
static inline cnt_t fmax(double a, cnt_t b) { return cnt_t(std::fmax(a, b.v)); }
static inline cnt_t fmin(cnt_t a, cnt_t b) { return cnt_t(std::fmin(a.v, b.v)); }
static inline cnt_t fmin(cnt_t a, double b) { return cnt_t(std::fmin(a.v, b)); }
static inline cnt_t fmin(double a, cnt_t b) { return cnt_t(std::fmin(a, b.v)); }
static inline bool isfinite(cnt_t a) { return std::isfinite(a.v); }

// the oracle, with every double a counted one (its system headers are already included);
// NAN and INFINITY become counted constants too, so that a conditional mixing them with a
// counted value has one type
#undef NAN
#undef INFINITY
#define NAN cnt_t(__builtin_nan(""))
#define INFINITY cnt_t(__builtin_inf())
#define double cnt_t
#include "m2c_oracle.c"
#undef double

namespace {

void reset() { std::memset(&opc::g, 0, sizeof(opc::g)); }
unsigned long long flops() { return opc::g.add + opc::g.mul + opc::g.div + opc::g.sqrt; }

void put(double* out) {
  out[0] = (double)opc::g.add;
  out[1] = (double)opc::g.mul;
  out[2] = (double)opc::g.div;
  out[3] = (double)opc::g.sqrt;
  out[4] = (double)opc::g.special;
}

}  // namespace

extern "C" {

// Counts of one call of each part of a time step, for the cell state P (rho,
// u, v, w, p) of material type/prm: out[k][0..4] = (add, mul, div, sqrt,
// special) of
//   k = 0: conservative -> primitive (cons_to_prim, without its sound-speed check)
//   k = 1: the sound speed check of cons_to_prim (eos_c2) alone
//   k = 2: one MUSCL face-state pair along an axis (5 limited slopes on data with
//          a b > 0, the two face states q -/+ sigma/2)
//   k = 3: one HLLC flux between the two face states (their e, c^2, c, E included)
//   k = 4: one third-order upwind level-set derivative
//   k = 5: one cell's reinitialisation update (away from the first layer), per iteration
int opc_parts(int type, const double* prm, const double* P, double out[6][5]) {
  or_eos_t q;
  mk_eos(&q, type, (const cnt_t*)prm);
  cnt_t Pc[5], W[5], Q[5];
  for (int v = 0; v < 5; ++v) Pc[v] = P[v];
  if (prim_to_cons(&q, Pc, W) != OR_OK) return 1;
  reset();
  if (cons_to_prim(&q, W, Q) != OR_OK) return 1;
  put(out[0]);
  cnt_t c2;
  reset();
  eos_c2(&q, Pc[0], Pc[4], &c2);
  put(out[1]);
  for (int v = 0; v < 5; ++v) out[0][v] -= out[1][v];
  // face states of a smooth profile along x: neighbours 1% below and above
  cnt_t Pm[5], Pp[5], Qm[5], Qp[5];
  for (int v = 0; v < 5; ++v) {
    const double s = (v >= 1 && v <= 3) ? (double)Pc[v] * 0.01 + 1.0 : (double)Pc[v] * 0.01;
    Pm[v] = (double)Pc[v] - s;
    Pp[v] = (double)Pc[v] + s;
  }
  reset();
  for (int v = 0; v < 5; ++v) {
    cnt_t a = Pc[v] - Pm[v], b = Pp[v] - Pc[v];
    cnt_t sg = va_slope(a, b);
    Qm[v] = Pc[v] - 0.5 * sg;
    Qp[v] = Pc[v] + 0.5 * sg;
  }
  // the subtractions forming a and b are part of the reconstruction: counted above
  put(out[2]);
  cnt_t F[5];
  reset();
  if (hllc(&q, Qp, Pp, 0, F) != OR_OK) return 1;
  put(out[3]);
  // level-set derivative on a 5-cell stencil (x axis of a 5 x 1 x 1 grid)
  or_grid_t g;
  std::memset(&g, 0, sizeof(g));
  g.n[0] = 5; g.n[1] = 1; g.n[2] = 1;
  g.h = 0.01;
  cnt_t phi[5] = {0.1, 0.11, 0.125, 0.14, 0.16};
  reset();
  ls_derivative(&g, phi, 2, 0, 0, 0, 3.0);
  put(out[4]);
  // reinitialisation: one iteration on an 8 x 8 x 8 grid with phi > 0 (no first layer), per cell
  g.n[0] = g.n[1] = g.n[2] = 8;
  g.reinit_every = 1;
  const long N = 512;
  cnt_t* ph = (cnt_t*)std::malloc(sizeof(cnt_t) * N * 3);
  for (long c = 0; c < N; ++c) ph[c] = 1.0 + 0.01 * (double)(c % 7) + 0.003 * (double)(c % 5);
  reset();
  reinit(&g, ph, 1, ph + N, ph + 2 * N);
  for (int k = 0; k < 5; ++k) out[5][k] = 0.0;
  put(out[5]);
  for (int k = 0; k < 5; ++k) out[5][k] /= (double)N;
  std::free(ph);
  return 0;
}

// Counts of one exact two-material Riemann solve and its two FIVER fluxes (an
// interface face), for side states wL, wR = (rho, u, p): out = (add, mul, div,
// sqrt, special), iters = the iteration count.
int opc_fiver_face(int typeL, const double* prmL, const double* wL, int typeR, const double* prmR,
                   const double* wR, double* out, int* iters) {
  or_eos_t qL, qR;
  mk_eos(&qL, typeL, (const cnt_t*)prmL);
  mk_eos(&qR, typeR, (const cnt_t*)prmR);
  cnt_t a[3] = {wL[0], wL[1], wL[2]}, b[3] = {wR[0], wR[1], wR[2]}, rs[4];
  reset();
  const int st = riemann(&qL, a, &qR, b, rs, iters);
  if (st) return st;
  cnt_t PL[5] = {a[0], a[1], 0.0, 0.0, a[2]}, PR[5] = {b[0], b[1], 0.0, 0.0, b[2]};
  cnt_t SL[5] = {rs[2], rs[1], 0.0, 0.0, rs[0]}, SR[5] = {rs[3], rs[1], 0.0, 0.0, rs[0]};
  cnt_t F[5];
  hllc(&qL, PL, SL, 0, F);
  hllc(&qR, SR, PR, 0, F);
  put(out);
  return 0;
}

}  // extern "C"
