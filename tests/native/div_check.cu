// Device check of the FP64 reciprocal and quotient of the bulk kernels
// (rcp_nr, div_nr) against the IEEE operations: random operands over the
// Newton range and beyond it, short mantissas, all-ones mantissas (the inputs
// where a faithful reciprocal may miss by an ulp), exact quotients, quotients
// that overflow or underflow (into the subnormal range and to zero) and signed
// zero numerators. Prints the number of quotients whose bits differ from
// a / b (NaNs compare equal) and the worst reciprocal error in ulps.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "m2c_physics.cuh"

__global__ void k_div(const double* a, const double* b, double* x, double* y, double* q, double* d, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    x[i] = m2c::rcp_nr(b[i]);
    y[i] = 1.0 / b[i];
    q[i] = m2c::div_nr(a[i], b[i]);
    d[i] = a[i] / b[i];
  }
}

// rsqrt_nr against the IEEE 1/sqrt(x) for positive x (a[i] taken positive)
__global__ void k_rsqrt(const double* a, double* r, double* s, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double x = fabs(a[i]);
    r[i] = m2c::rsqrt_nr(x);
    s[i] = 1.0 / sqrt(x);
  }
}

static double ulps(double v, double r) {
  if (v == r) return 0.0;
  if (std::isnan(v) && std::isnan(r)) return 0.0;
  return std::fabs(v - r) / (std::nextafter(std::fabs(r), INFINITY) - std::fabs(r));
}

int main() {
  const int n = 1 << 20;
  std::mt19937_64 g(20250822);
  double *ha = new double[n], *hb = new double[n], *hx = new double[n], *hy = new double[n], *hq = new double[n],
         *hd = new double[n];
  for (int i = 0; i < n; ++i) {
    hb[i] = std::ldexp(1.0 + (double)(g() >> 11) * 0x1p-53, (int)(g() % 280) - 140) * ((g() & 1) ? -1.0 : 1.0);
    ha[i] = std::ldexp(1.0 + (double)(g() >> 11) * 0x1p-53, (int)(g() % 200) - 100) * ((g() & 1) ? -1.0 : 1.0);
    if (i % 8 == 1) hb[i] = std::ldexp(1.0 + (double)(g() % 64) / 64.0, (int)(g() % 40) - 20);
    if (i % 8 == 2) hb[i] = std::nextafter(std::ldexp(1.0, (int)(g() % 40) - 19), 0.0);
    if (i % 8 == 3) ha[i] = hb[i] * (double)(g() % 1000);
    if (i % 16 == 4) ha[i] = std::ldexp(1.0 + (double)(g() >> 11) * 0x1p-53, 880 + (int)(g() % 143));
    if (i % 16 == 12) ha[i] = std::ldexp(1.0 + (double)(g() >> 11) * 0x1p-53, -1074 + (int)(g() % 200));
    if (i % 16 == 5) ha[i] = (g() & 1) ? 0.0 : -0.0;
  }
  ha[7] = 1e308; hb[7] = 0.5;    // overflows to infinity
  ha[8] = -1e308; hb[8] = 1e-30;
  ha[9] = 1e-300; hb[9] = 1e30;  // subnormal quotient
  ha[10] = 4.9e-324; hb[10] = 3.0;
  ha[11] = -0.0; hb[11] = 7.0;   // signed zeros
  ha[12] = 0.0; hb[12] = -7.0;
  ha[13] = INFINITY; hb[13] = 2.0;
  ha[14] = NAN; hb[14] = 2.0;
  hb[0] = 0.0; hb[1] = -0.0; hb[2] = INFINITY; hb[3] = NAN; hb[4] = 0x1p-125; hb[5] = 0x1p125; hb[6] = 1e-300;
  double *da, *db, *dx, *dy, *dq, *dd;
  const size_t bytes = sizeof(double) * n;
  if (cudaMalloc(&da, bytes) || cudaMalloc(&db, bytes) || cudaMalloc(&dx, bytes) || cudaMalloc(&dy, bytes) ||
      cudaMalloc(&dq, bytes) || cudaMalloc(&dd, bytes)) {
    printf("cudaMalloc failed\n");
    return 1;
  }
  cudaMemcpy(da, ha, bytes, cudaMemcpyHostToDevice);
  cudaMemcpy(db, hb, bytes, cudaMemcpyHostToDevice);
  k_div<<<(n + 255) / 256, 256>>>(da, db, dx, dy, dq, dd, n);
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    printf("kernel failed: %s\n", cudaGetErrorString(e));
    return 1;
  }
  cudaMemcpy(hx, dx, bytes, cudaMemcpyDeviceToHost);
  cudaMemcpy(hy, dy, bytes, cudaMemcpyDeviceToHost);
  cudaMemcpy(hq, dq, bytes, cudaMemcpyDeviceToHost);
  cudaMemcpy(hd, dd, bytes, cudaMemcpyDeviceToHost);
  long ndiv = 0;
  double worst_rcp = 0.0;
  for (int i = 0; i < n; ++i) {
    const bool same = std::memcmp(&hq[i], &hd[i], sizeof(double)) == 0 || (std::isnan(hq[i]) && std::isnan(hd[i]));
    if (!same) ++ndiv;
    const double u = ulps(hx[i], hy[i]);
    if (!(u <= worst_rcp)) worst_rcp = u;
  }
  k_rsqrt<<<(n + 255) / 256, 256>>>(db, dx, dy, n);  // reuses the x, y buffers
  const cudaError_t e2 = cudaDeviceSynchronize();
  if (e2 != cudaSuccess) {
    printf("kernel failed: %s\n", cudaGetErrorString(e2));
    return 1;
  }
  cudaMemcpy(hx, dx, bytes, cudaMemcpyDeviceToHost);
  cudaMemcpy(hy, dy, bytes, cudaMemcpyDeviceToHost);
  double worst_rsqrt = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!(std::fabs(hb[i]) > 0.0) || !std::isfinite(hb[i])) continue;
    const double u = ulps(hx[i], hy[i]);
    if (!(u <= worst_rsqrt)) worst_rsqrt = u;
  }
  printf("quotient mismatches %ld\nreciprocal worst ulp %g\nrsqrt worst ulp %g\n", ndiv, worst_rcp,
         worst_rsqrt);
  return 0;
}
