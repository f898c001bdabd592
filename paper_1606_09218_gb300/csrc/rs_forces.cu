// Forces from the discrete gradient of the RS-Tucker tensor (Sec. 4.3, Eq. (4.9)).
//
// The discrete gradient applies a one-dimensional difference operator D_h to one mode of every
// term.  For the Tucker form of the long-range part (Def. 3.9) the mode-l derivative is the core
// contracted with the differentiated basis D_h V_l instead of V_l, so at a grid point
//   d1 P_l^T(i) = sum_ab (D_h V1)[i1][a] V2[i2][b] T1[a][b][i3]
//   d2 P_l^T(i) = sum_ab V1[i1][a] (D_h V2)[i2][b] T1[a][b][i3]
//   d3 P_l^T(i) = sum_ab V1[i1][a] V2[i2][b] T1d[a][b][i3]
// with T1 = beta x_3 V3 and T1d = beta x_3 (D_h V3), both formed here in i3-major layout.
// The force on particle j is F_j = -z_j [grad_h P_l^T(x_j) - z_j grad_h K_l(0)] minus the
// window gradients of the other particles (term by term, as in the pair path), the particle's
// own long-range term taken out (its centred difference is zero; a one-sided row near the ends
// of the grid gives it a small value).  O(N r1 r2) work after the O(n r) differences and one
// r^2 x n x r product, instead of O(N^2 R_l) for the pair kernel.
//
// D_h: the centred first-derivative formula of order FD_ORDER in the interior, the same number
// of points shifted into the grid near its ends; the weights come from Fornberg's recurrence
// (B. Fornberg, "Generation of finite difference formulas on arbitrarily spaced grids",
// Math. Comp. 51 (1988) 699-706) evaluated in double precision on the host.
#include "rs_internal.cuh"

#include <cmath>
#include <vector>

namespace rs {

namespace {

// Weights of the first derivative at 0 from the values at the integer offsets x[0..m-1]
// (Fornberg's recurrence for derivative orders 0 and 1); w[i] multiplies f(x[i] h) / h.
void fornberg_first_derivative(const double* x, int m, double* w) {
  std::vector<double> c0(m, 0.0), c1(m, 0.0);     // weights of the 0th and 1st derivative
  double a1 = 1.0;
  double a4 = x[0];
  c0[0] = 1.0;
  for (int i = 1; i < m; ++i) {
    double a2 = 1.0;
    const double a5 = a4;
    a4 = x[i];
    for (int j = 0; j < i; ++j) {
      const double a3 = x[i] - x[j];
      a2 *= a3;
      if (j == i - 1) {
        c1[i] = a1 * (c0[i - 1] - a5 * c1[i - 1]) / a2;
        c0[i] = -a1 * a5 * c0[i - 1] / a2;
      }
      c1[j] = (a4 * c1[j] - c0[j]) / a3;
      c0[j] = a4 * c0[j] / a3;
    }
    a1 = a2;
  }
  for (int i = 0; i < m; ++i) w[i] = c1[i];
}

}  // namespace

bool fd_table(int n, double h, double* w, int* start) {
  if (n < 2 || !(h > 0.0)) return false;
  const int width = n < FD_WIDTH ? n : FD_WIDTH;
  double x[FD_WIDTH], wt[FD_WIDTH];
  for (int i = 0; i < n; ++i) {
    int s = i - width / 2;
    if (s < 0) s = 0;
    if (s > n - width) s = n - width;
    for (int q = 0; q < width; ++q) x[q] = (double)(s + q - i);
    fornberg_first_derivative(x, width, wt);
    for (int q = 0; q < FD_WIDTH; ++q) w[(size_t)i * FD_WIDTH + q] = q < width ? wt[q] / h : 0.0;
    start[i] = s;
  }
  return true;
}

// dZ[l][i][a] = sum_q w[i][q] Z[l][start[i] + q][a] for a < rank[l], zero for the other columns
// (FP64, with an FP32 copy for the bulk path).  Grid (n, 3), threads over a.
__global__ void fd_basis_kernel(const double* __restrict__ Z64, const double* __restrict__ w,
                                const int* __restrict__ start, int n, int rmax, const DevScalars* sc,
                                double* dZ64, float* dZ32) {
  const int i = blockIdx.x, l = blockIdx.y;
  const int r = sc->rank[l];
  const double* Zl = Z64 + (long long)l * n * rmax;
  const int s = start[i];
  for (int a = threadIdx.x; a < rmax; a += blockDim.x) {
    double v = 0.0;
    if (a < r) {
#pragma unroll
      for (int q = 0; q < FD_WIDTH; ++q) {
        const double wq = w[(long long)i * FD_WIDTH + q];
        if (wq != 0.0) v = fma(wq, Zl[(long long)(s + q) * rmax + a], v);
      }
    }
    const long long o = ((long long)l * n + i) * rmax + a;
    dZ64[o] = v;
    dZ32[o] = (float)v;
  }
}

template <typename T> struct FdBulk;
template <> struct FdBulk<float> {
  static const float* Z(const Ctx& c) { return c.Z32; }
  static const float* dZ(const Ctx& c) { return c.dZ32; }
};
template <> struct FdBulk<double> {
  static const double* Z(const Ctx& c) { return c.Z64; }
  static const double* dZ(const Ctx& c) { return c.dZ64; }
};

// One warp per charged particle: the three differentiated Tucker values at its grid point (the
// lanes share the (a, b) pairs; products of T, sums in FP64), its own term's difference, and the
// window gradients of the other particles; F = -z (grad - z grad_self).  Particles without
// charge keep the zero force of the memset.  T1, T1d: the slices [i3][a][b] (leading size rmax^2).
template <typename T>
__global__ void __launch_bounds__(256)
forces_rs_kernel(DevView c, const T* __restrict__ Zb, const T* __restrict__ dZb, const T* __restrict__ T1,
                 const T* __restrict__ T1d, const double* __restrict__ dpk64, const double* __restrict__ fw,
                 const int* __restrict__ fs, double* Fout) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m = blockIdx.x * 8 + warp;
  const int nnz = c.sc->n_nz;
  if (m >= nnz) return;
  const int p = c.nz_idx[m];
  const int n = c.n, rmax = c.rmax, L = 2 * n - 1;
  const int i1 = c.j[3 * p], i2 = c.j[3 * p + 1], i3 = c.j[3 * p + 2];
  const int r1 = c.sc->rank[0], r2 = c.sc->rank[1];
  const long long sZ = (long long)n * rmax;
  const T* V1 = Zb + (long long)i1 * rmax;
  const T* V2 = Zb + sZ + (long long)i2 * rmax;
  const T* D1 = dZb + (long long)i1 * rmax;
  const T* D2 = dZb + sZ + (long long)i2 * rmax;
  double g1 = 0.0, g2 = 0.0, g3 = 0.0;
  const T* S = T1 + (long long)i3 * rmax * rmax;      // slices at i3 ([a][b], i3-major layout)
  const T* Sd = T1d + (long long)i3 * rmax * rmax;
  for (int e = lane; e < r1 * r2; e += 32) {
    const int a = e / r2, b = e % r2;
    const long long o = (long long)a * rmax + b;
    const double t = (double)S[o], td = (double)Sd[o];
    const double u = (double)V1[a], ud = (double)D1[a], v = (double)V2[b], vd = (double)D2[b];
    g1 += ud * v * t;
    g2 += u * vd * t;
    g3 += u * v * td;
  }
  // the particle's own long-range term: D_h along mode l of sum_k p_k(. - j) at j
  {
    const double z = c.Z[p];
    for (int e = lane; e < 3 * FD_WIDTH; e += 32) {
      const int l = e / FD_WIDTH, q = e % FD_WIDTH;
      const int il = l == 0 ? i1 : (l == 1 ? i2 : i3);
      const double wq = fw[(long long)il * FD_WIDTH + q];
      if (wq == 0.0) continue;
      const int d = fs[il] + q - il;
      double s = 0.0;
      for (int k = 0; k < c.R_l; ++k) {
        const double* row = c.pk64 + (long long)k * L + n - 1;
        s += row[d] * row[0] * row[0];
      }
      const double v = z * wq * s;
      if (l == 0) g1 -= v;
      else if (l == 1) g2 -= v;
      else g3 -= v;
    }
  }
  window_grad_add(c, dpk64, i1, i2, i3, p, lane, g1, g2, g3);
  for (int o = 16; o > 0; o >>= 1) {
    g1 += __shfl_down_sync(0xffffffffu, g1, o);
    g2 += __shfl_down_sync(0xffffffffu, g2, o);
    g3 += __shfl_down_sync(0xffffffffu, g3, o);
  }
  if (lane == 0) {
    const double z = c.Z[p];
    Fout[3 * p] = -z * g1;
    Fout[3 * p + 1] = -z * g2;
    Fout[3 * p + 2] = -z * g3;
  }
}

template <typename T>
static int forces_rs_t(Ctx& c) {
  const int n = c.n, rmax = c.rmax;
  fd_basis_kernel<<<dim3(n, 3), 128, 0, c.stream>>>(c.Z64, c.fd_w, c.fd_s, n, rmax, c.sc, c.dZ64, c.dZ32);
  // the slices of T1 = beta x_3 V3 and T1d = beta x_3 (D_h V3) at one grid index i3, laid out
  // i3-major ([i3][a][b], two row blocks of T1d) so that the lanes of a warp read consecutive b:
  //   T1d[i3][(a, b)] = sum_c V3[i3][c] beta[(a, b)][c],  T1d[n + i3][(a, b)] = sum_c (D_h V3)[i3][c] beta[(a, b)][c]
  const long long sZ = (long long)n * rmax;
  const long long slab = (long long)n * rmax * rmax;
  gemm_batched<T>(c.stream, false, true, n, rmax * rmax, rmax, T(1), FdBulk<T>::Z(c) + 2 * sZ, rmax, 0,
                  (const T*)c.beta, rmax, 0, T(0), (T*)c.T1d, rmax * rmax, 0, 1, nullptr, nullptr, c.sc->rank + 2,
                  &c.gscr);
  gemm_batched<T>(c.stream, false, true, n, rmax * rmax, rmax, T(1), FdBulk<T>::dZ(c) + 2 * sZ, rmax, 0,
                  (const T*)c.beta, rmax, 0, T(0), (T*)c.T1d + slab, rmax * rmax, 0, 1, nullptr, nullptr,
                  c.sc->rank + 2, &c.gscr);
  cudaMemsetAsync(c.Fout, 0, sizeof(double) * 3 * (size_t)c.maxN, c.stream);
  int blocks = (c.maxN + 7) / 8;
  if (blocks < 1) blocks = 1;
  forces_rs_kernel<T><<<blocks, 256, 0, c.stream>>>(make_view(c), FdBulk<T>::Z(c), FdBulk<T>::dZ(c),
                                                    (const T*)c.T1d, (const T*)c.T1d + slab, c.dpk64, c.fd_w,
                                                    c.fd_s, c.Fout);
  return 4;
}

int launch_forces_rs(Ctx& c) { return c.fp64 ? forces_rs_t<double>(c) : forces_rs_t<float>(c); }

}  // namespace rs
