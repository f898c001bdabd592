// Plain-method GPU paths: the same potential on the same grid without the RS format, the
// comparisons of the RS path on one GPU.
//
//  * direct sum (Sec. 1, Eq. (1.1)):  P[i] = sum_nu z_nu / |x_i - x_nu|, n^3 N pair terms
//    (terms with |x_i - x_nu| = 0 skipped);
//  * full-rank canonical sum (Eq. (3.4) with all R quadrature terms, no split, no truncation):
//    P_0[i] = sum_nu z_nu sum_k p_k[i1 - j1] p_k[i2 - j2] p_k[i3 - j3], 2 n^3 N R operations.
//
// Both at the snapped centres x_nu = -b + j_nu h of the last solve of a context, products and
// square roots in FP32, every output's sum compensated (32-term FP32 chunks folded into an
// FP32 (hi, lo) pair by an error-free two-sum), so the results carry about 1e-7 relative error.
#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr int PD_THREADS = 128;              // direct sum: one CTA per grid row (i1, i2)
constexpr int PD_PTS = 5;                    // i3 points of a thread (n <= 640 in one pass)
constexpr int PD_CHUNK = 1024;               // particles staged in shared memory at a time
constexpr int PC_THREADS = 256;              // canonical sum: one CTA per 4 columns (i2, i3..i3+3)
constexpr int PC_ROWS = 5;                   // i1 rows of a thread (n <= 1280 in one pass)
constexpr int PC_TERMS = 256;                // (particle, k) terms staged at a time

__device__ __forceinline__ void fold(float& hi, float& lo, float& acc) {
  const float s = hi + acc;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (acc - bp);
  hi = s;
  acc = 0.f;
}

}  // namespace

__global__ void __launch_bounds__(PD_THREADS)
plain_direct_kernel(const int* __restrict__ jidx, const int* __restrict__ nz_idx, const double* __restrict__ Z,
                    const DevScalars* sc, int n, float b, float h, float* __restrict__ out) {
  __shared__ float4 sp[PD_CHUNK];
  const int i1 = blockIdx.x / n, i2 = blockIdx.x % n;
  const float x1 = -b + h * (float)i1, x2 = -b + h * (float)i2;
  const int nnz = sc->n_nz;
  float acc[PD_PTS], hi[PD_PTS], lo[PD_PTS], x3[PD_PTS];
#pragma unroll
  for (int q = 0; q < PD_PTS; ++q) {
    acc[q] = hi[q] = lo[q] = 0.f;
    x3[q] = -b + h * (float)(threadIdx.x + q * PD_THREADS);
  }
  int cnt = 0;
  for (int m0 = 0; m0 < nnz; m0 += PD_CHUNK) {
    __syncthreads();
    for (int e = threadIdx.x; e < PD_CHUNK; e += PD_THREADS) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m0 + e < nnz) {
        const int p = nz_idx[m0 + e];
        const float X = -b + h * (float)jidx[3 * p], Y = -b + h * (float)jidx[3 * p + 1];
        const float dx = x1 - X, dy = x2 - Y;
        v = make_float4(fmaf(dx, dx, dy * dy), -b + h * (float)jidx[3 * p + 2], (float)Z[p], 0.f);
      }
      sp[e] = v;
    }
    __syncthreads();
    const int lim = min(PD_CHUNK, nnz - m0);
    for (int e = 0; e < lim; ++e) {
      const float4 v = sp[e];
#pragma unroll
      for (int q = 0; q < PD_PTS; ++q) {
        const float dz = x3[q] - v.y;
        const float r2 = fmaf(dz, dz, v.x);
        acc[q] += r2 > 0.f ? v.z * rsqrtf(r2) : 0.f;
      }
      if (++cnt == 32) {
#pragma unroll
        for (int q = 0; q < PD_PTS; ++q) fold(hi[q], lo[q], acc[q]);
        cnt = 0;
      }
    }
  }
  const long long row = ((long long)i1 * n + i2) * n;
#pragma unroll
  for (int q = 0; q < PD_PTS; ++q) {
    fold(hi[q], lo[q], acc[q]);
    const int i3 = threadIdx.x + q * PD_THREADS;
    if (i3 < n) out[row + i3] = hi[q] + lo[q];
  }
}

__global__ void __launch_bounds__(PC_THREADS)
plain_canonical_kernel(const float* __restrict__ pk, const int* __restrict__ jidx,
                       const int* __restrict__ nz_idx, const double* __restrict__ Z, const DevScalars* sc,
                       int n, int R, float* __restrict__ out) {
  extern __shared__ __align__(16) float pc_smem[];
  float* tab = pc_smem;                                   // R x (2n - 1) factors
  float4* w = (float4*)(tab + (((size_t)R * (2 * n - 1) + 3) & ~(size_t)3));   // [PC_TERMS] weights
  int* j1 = (int*)(w + PC_TERMS);                         // [PC_TERMS] row offsets k L + j1
  const int L = 2 * n - 1;
  const int ntile = (n + 3) / 4;
  const int i2 = blockIdx.x / ntile, i3a = (blockIdx.x % ntile) * 4;
  for (int e = threadIdx.x; e < R * L; e += PC_THREADS) tab[e] = pk[e];
  const int nnz = sc->n_nz;
  const long long T = (long long)nnz * R;
  float acc[PC_ROWS][4], hi[PC_ROWS][4], lo[PC_ROWS][4];
#pragma unroll
  for (int r = 0; r < PC_ROWS; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = hi[r][c] = lo[r][c] = 0.f;
  const int nrows = (n + PC_THREADS - 1) / PC_THREADS;  // i1 rows in use (<= PC_ROWS)
  int cnt = 0;
  for (long long t0 = 0; t0 < T; t0 += PC_TERMS) {
    __syncthreads();
    {
      // weights z p_k[i2 - j2] p_k[i3 - j3] of this block's four columns
      const long long t = t0 + threadIdx.x;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      int off = 0;
      if (t < T) {
        const int p = nz_idx[t / R], k = (int)(t % R);
        const float* row = tab + (size_t)k * L + (n - 1);
        const float zf = (float)Z[p] * row[i2 - jidx[3 * p + 1]];
        const int d3 = i3a - jidx[3 * p + 2];
        v.x = zf * row[d3];
        v.y = (i3a + 1 < n) ? zf * row[d3 + 1] : 0.f;
        v.z = (i3a + 2 < n) ? zf * row[d3 + 2] : 0.f;
        v.w = (i3a + 3 < n) ? zf * row[d3 + 3] : 0.f;
        off = k * L + (n - 1) - jidx[3 * p];
      }
      w[threadIdx.x] = v;
      j1[threadIdx.x] = off;
    }
    __syncthreads();
    const int lim = (int)min((long long)PC_TERMS, T - t0);
    for (int e = 0; e < lim; ++e) {
      const float4 v = w[e];
      const float* f = tab + j1[e];
#pragma unroll
      for (int r = 0; r < PC_ROWS; ++r) {
        if (r < nrows) {
          const int i1 = threadIdx.x + r * PC_THREADS;
          const float p1 = i1 < n ? f[i1] : 0.f;
          acc[r][0] = fmaf(v.x, p1, acc[r][0]);
          acc[r][1] = fmaf(v.y, p1, acc[r][1]);
          acc[r][2] = fmaf(v.z, p1, acc[r][2]);
          acc[r][3] = fmaf(v.w, p1, acc[r][3]);
        }
      }
      if (++cnt == 32) {
#pragma unroll
        for (int r = 0; r < PC_ROWS; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) fold(hi[r][c], lo[r][c], acc[r][c]);
        cnt = 0;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < PC_ROWS; ++r) {
    const int i1 = threadIdx.x + r * PC_THREADS;
    if (i1 >= n) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      fold(hi[r][c], lo[r][c], acc[r][c]);
      if (i3a + c < n) out[((long long)i1 * n + i2) * n + i3a + c] = hi[r][c] + lo[r][c];
    }
  }
}

size_t plain_canonical_smem(const Ctx& c) {
  return sizeof(float) * (((size_t)c.R * (2 * c.n - 1) + 3) & ~(size_t)3) + sizeof(float4) * PC_TERMS +
         sizeof(int) * PC_TERMS;
}

rs_status launch_plain(Ctx& c, int which, float* out) {
  if (which == 0) {
    if (c.n > PD_THREADS * PD_PTS) return RS_ERR_CAPACITY;
    plain_direct_kernel<<<(unsigned)((long long)c.n * c.n), PD_THREADS, 0, c.stream>>>(
        c.j, c.nz_idx, c.Z, c.sc, c.n, (float)c.cfg.b, (float)c.h, out);
  } else {
    if (c.n > PC_THREADS * PC_ROWS) return RS_ERR_CAPACITY;
    const size_t shm = plain_canonical_smem(c);
    if (shm > 227 * 1024) return RS_ERR_CAPACITY;
    const long long blocks = (long long)c.n * ((c.n + 3) / 4);
    plain_canonical_kernel<<<(unsigned)blocks, PC_THREADS, shm, c.stream>>>(c.pk32, c.j, c.nz_idx, c.Z, c.sc,
                                                                            c.n, c.R, out);
  }
  return RS_OK;
}

cudaError_t set_attributes_plain(int optin) {
  return allow_max_dynamic_smem((const void*)plain_canonical_kernel, optin);
}

}  // namespace rs
