// Energy and forces at centres off the grid (the FP32 bulk workload with finite-difference
// checks, h = 1e-4 far below the grid spacing): the RS kernel of the context in pair form,
//
//   E = 1/2 sum_{j != nu} z_j z_nu K_h(x_j - x_nu),   K_h(r) = sum_{k < R} p_k(r1) p_k(r2) p_k(r3),
//   F_j = -dE/dx_j = -z_j sum_{nu != j} z_nu grad K_h(x_j - x_nu)                   (Sec. 4.2, 4.3)
//
// with p_k(y) = a_k^{1/3} (cell average of exp(-t_k^2 x^2) over the cell of width h centred at
// y), the Galerkin factors of Eq. (2.10) continued to any offset, and their derivative
// a_k^{1/3} (exp(-t_k^2 (y + h/2)^2) - exp(-t_k^2 (y - h/2)^2)) / h.  On grid offsets this is
// exactly the kernel of the RS grid tensor; off the grid it is smooth in the centres, so its
// gradient is the adjoint of the energy.  All pairs and all R terms (no cut-off: a window
// radius would make E jump when a pair crosses it).
//
// Precision: offsets in FP64, factors in FP32 (relative 1e-7), sums in FP64.  With m = t y and
// d = t h / 2 the cell average is sqrt(pi) (erf(m + d) - erf(m - d)) / (4 d).  Where the
// Gaussian hardly changes over the cell (d < 0.1 and |m| d < 0.025) it is taken by three-point
// Gauss-Legendre quadrature, 1/2 sum_i w_i exp(-(m + d xi_i)^2), free of the cancellation of the
// difference (the rule's error term, of order (2 m d)^6 and d^6, is below 1e-10 there);
// elsewhere by the erf difference (erfc in the tail), which then loses at most one digit.  The
// derivative's exp(-b^2) - exp(-a^2) is -2 exp(-(m^2 + d^2)) sinh(2 m d) for 2 |m| d < 1.
#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr int PF_WARPS = 8;
constexpr int PF_RMAX = 64;

__device__ __forceinline__ float cell_avg(float m, float d) {
  if (d < 0.1f && fabsf(m) * d < 0.025f) {
    const float xi = 0.7745966692414834f;          // sqrt(3/5)
    const float u0 = m - d * xi, u1 = m, u2 = m + d * xi;
    return 0.5f * ((5.f / 9.f) * expf(-u0 * u0) + (8.f / 9.f) * expf(-u1 * u1) +
                   (5.f / 9.f) * expf(-u2 * u2));
  }
  const float a = fabsf(m) - d, b = fabsf(m) + d;  // the average is even in m
  const float diff = (a > 0.5f) ? (erfcf(a) - erfcf(b)) : (erff(b) - erff(a));
  return 0.4431134627263791f * diff / d;             // sqrt(pi) / 4 * (erf(b) - erf(a)) / d
}

// exp(-(m + d)^2) - exp(-(m - d)^2): as -2 exp(-(m^2 + d^2)) sinh(2 m d) while 2 |m| d < 1
// (no cancellation), as the difference itself beyond (no overflow of sinh; the two terms then
// differ by at least e^2)
__device__ __forceinline__ float cell_avg_diff(float m, float d) {
  const float x = 2.f * m * d;
  if (fabsf(x) < 1.f) return -2.f * expf(-(m * m + d * d)) * sinhf(x);
  return expf(-(m + d) * (m + d)) - expf(-(m - d) * (m - d));
}

}  // namespace

// one warp per particle j (charged); lanes over the other charged particles
__global__ void __launch_bounds__(32 * PF_WARPS)
pair_energy_forces_kernel(const double* __restrict__ xyz, const double* __restrict__ Z, int N, int R,
                          double h, double hq, double u0, double* __restrict__ pe, double* __restrict__ F) {
  __shared__ float st[PF_RMAX], sa[PF_RMAX];        // t_k, a_k
  if (threadIdx.x < R) {
    const double t = exp(u0 + threadIdx.x * hq);
    st[threadIdx.x] = (float)t;
    sa[threadIdx.x] = (float)(1.1283791670955126 * hq * t);   // (2 / sqrt(pi)) h_q t_k
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * PF_WARPS + warp;
  if (j >= N) return;
  const double zj = Z[j];
  double e = 0.0, f0 = 0.0, f1 = 0.0, f2 = 0.0;
  if (zj != 0.0) {
    const double x0 = xyz[3 * j], x1 = xyz[3 * j + 1], x2 = xyz[3 * j + 2];
    const float hf = (float)h, ih = (float)(1.0 / h);
    for (int nu = lane; nu < N; nu += 32) {
      const double zn = Z[nu];
      if (nu == j || zn == 0.0) continue;
      const double y0 = x0 - xyz[3 * nu], y1 = x1 - xyz[3 * nu + 1], y2 = x2 - xyz[3 * nu + 2];
      float K = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
      for (int k = 0; k < R; ++k) {
        const float t = st[k], d = 0.5f * t * hf;
        const float m0 = (float)(y0 * t), m1 = (float)(y1 * t), m2 = (float)(y2 * t);
        const float c0 = cell_avg(m0, d), c1 = cell_avg(m1, d), c2 = cell_avg(m2, d);
        // derivatives of the cell averages in the offset: (exp(-b^2) - exp(-a^2)) / h
        const float q0 = cell_avg_diff(m0, d) * ih;
        const float q1 = cell_avg_diff(m1, d) * ih;
        const float q2 = cell_avg_diff(m2, d) * ih;
        const float s = sa[k];                       // a_k (three factors of a_k^{1/3})
        K = fmaf(s, c0 * c1 * c2, K);
        g0 = fmaf(s, q0 * c1 * c2, g0);
        g1 = fmaf(s, c0 * q1 * c2, g1);
        g2 = fmaf(s, c0 * c1 * q2, g2);
      }
      e += zn * (double)K;
      f0 += zn * (double)g0;
      f1 += zn * (double)g1;
      f2 += zn * (double)g2;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, o);
    f0 += __shfl_down_sync(0xffffffffu, f0, o);
    f1 += __shfl_down_sync(0xffffffffu, f1, o);
    f2 += __shfl_down_sync(0xffffffffu, f2, o);
  }
  if (lane == 0) {
    pe[j] = 0.5 * zj * e;
    if (F) {
      F[3 * j] = -zj * f0;
      F[3 * j + 1] = -zj * f1;
      F[3 * j + 2] = -zj * f2;
    }
  }
}

// E = sum_j pe[j] in a fixed order (one CTA)
__global__ void __launch_bounds__(1024) pair_energy_sum_kernel(const double* __restrict__ pe, int N, double* E) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += pe[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *E = v;
  }
}

rs_status launch_pair_energy_forces(Ctx& c, int N, const double* xyz, const double* Z, double* E, double* F) {
  if (c.R > PF_RMAX) return RS_ERR_INVALID_ARG;
  const int blocks = (N + PF_WARPS - 1) / PF_WARPS;
  if (N > 0)
    pair_energy_forces_kernel<<<blocks, 32 * PF_WARPS, 0, c.stream>>>(xyz, Z, N, c.R, c.h, c.cfg.h_q, c.cfg.u0,
                                                                      c.pe, F);
  pair_energy_sum_kernel<<<1, 1024, 0, c.stream>>>(c.pe, N, E);
  return RS_OK;
}

}  // namespace rs
