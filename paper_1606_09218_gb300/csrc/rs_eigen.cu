// Eigen stage of the RHOSVD (Sec. 6, step (I)): dominant left singular subspace of each
// long-range side matrix U^(l), computed from its Gram matrix G_l = U^(l) U^(l)^T.
//
//   X = G * Omega                      FP64, Omega a seeded Gaussian block (range finder)
//   Q = orth(X)                        FP64 block Gram-Schmidt (8 columns, two passes, Cholesky
//                                      QR inside blocks); stops where a block falls to rounding
//   T = Q^T G Q                        FP64 Rayleigh quotient
//   T -> W^T T W  (twice)              FP32 two-sided Jacobi on the graded T, rotations applied
//                                      and re-orthonormalised (Newton-Schulz) in FP64
//   ranks from diag(T) and trace(G)    tail(r) = trace(G) - trace(T) + sum_{i>=r} lambda_i
//
// FP64 keeps the small eigenvalues (down to eps^2 * trace) that the truncation needs; the
// FP32 Jacobi is accurate in the relative sense because T is graded after the FP64 steps.
#include "rs_internal.cuh"

#include <cstdio>
#include <cstdlib>
#include <utility>

namespace rs {

// ------------------------------------------------------------------ generic GEMM
template <typename T>
__global__ void __launch_bounds__(256)
gemm_kernel(bool tA, bool tB, int M, int N, int K, T alpha, const T* __restrict__ A, int lda,
            long long sA, const T* __restrict__ B, int ldb, long long sB, T beta, T* C, int ldc,
            long long sC, const int* dynM, const int* dynN, const int* dynK) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int bz = blockIdx.z;
  int m = M, nn = N, kk = K;
  if (dynM) m = min(m, dynM[bz]);
  if (dynN) nn = min(nn, dynN[bz]);
  if (dynK) kk = min(kk, dynK[bz]);
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  if (row0 >= m || col0 >= nn) return;
  const int kbeg = 0, kend = kk;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) acc[i][jj] = T(0);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + e * 256;
      int r, k;
      if (!tA) { r = idx / BK; k = idx % BK; } else { k = idx / BM; r = idx % BM; }
      int gr = row0 + r, gk = k0 + k;
      T v = T(0);
      if (gr < m && gk < kend) v = tA ? A[(long long)gk * lda + gr] : A[(long long)gr * lda + gk];
      As[k][r] = v;
      int c;
      if (!tB) { k = idx / BN; c = idx % BN; } else { c = idx / BK; k = idx % BK; }
      int gc = col0 + c;
      gk = k0 + k;
      T w = T(0);
      if (gc < nn && gk < kend) w = tB ? B[(long long)gc * ldb + gk] : B[(long long)gk * ldb + gc];
      Bs[k][c] = w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) bb[jj] = Bs[k][tx + 16 * jj];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(a[i], bb[jj], acc[i][jj]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gr = row0 + ty + 16 * i;
    if (gr >= m) continue;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      int gc = col0 + tx + 16 * jj;
      if (gc >= nn) continue;
      T* p = C + (long long)gr * ldc + gc;
      T v = alpha * acc[i][jj];
      if (beta != T(0)) v += beta * *p;
      *p = v;
    }
  }
}

// 16x16-tile kernel of the FP64 products: one output per thread, K split across CTAs so that
// the few FP64 units of every SM take part (GB300 issues about one FP64 FMA per clock and SM, so
// a 64x64 tile alone would take tens of microseconds).  The split is deterministic: every CTA
// stores its partial tile, and the last CTA of the tile to finish (counted with an atomic, after
// a fence) adds the partials in the order of their K ranges and writes C, so the result does not
// depend on the order in which the CTAs ran.  Entries of the M x N block outside the dynamic
// sizes are written as zero.
template <typename T>
__global__ void __launch_bounds__(256)
gemm_small_kernel(bool tA, bool tB, int M, int N, int K, T alpha, const T* __restrict__ A, int lda,
                  long long sA, const T* __restrict__ B, int ldb, long long sB, T* C, int ldc,
                  long long sC, int splitK, const int* dynM, const int* dynN, const int* dynK,
                  T* part, unsigned* count) {
  constexpr int BT = 16;
  __shared__ T As[BT][BT + 1];
  __shared__ T Bs[BT][BT + 1];
  __shared__ unsigned s_last;
  const int bz = blockIdx.z / splitK, kz = blockIdx.z % splitK;
  int m = M, nn = N, kk = K;
  if (dynM) m = min(m, dynM[bz]);
  if (dynN) nn = min(nn, dynN[bz]);
  if (dynK) kk = min(kk, dynK[bz]);
  const int row0 = blockIdx.y * BT, col0 = blockIdx.x * BT;
  const int tx = threadIdx.x % BT, ty = threadIdx.x / BT;
  const int gr = row0 + ty, gc = col0 + tx;
  C += bz * sC;
  if (row0 >= m || col0 >= nn) {                 // the whole tile is outside the dynamic sizes
    if (kz == 0 && gr < M && gc < N) C[(long long)gr * ldc + gc] = T(0);
    return;
  }
  const int chunk = ((kk + splitK - 1) / splitK + BT - 1) / BT * BT;
  const int kbeg = kz * chunk, kend = min(kk, kbeg + chunk);
  A += bz * sA;
  B += bz * sB;
  T acc = T(0);
  for (int k0 = kbeg; k0 < kend; k0 += BT) {
    {
      // consecutive threads read consecutive addresses: a transposed operand is loaded along its
      // rows and stored transposed in shared memory
      if (!tA) {
        const int ar = row0 + ty, gk = k0 + tx;            // A element (ar, gk)
        As[ty][tx] = (ar < m && gk < kend) ? A[(long long)ar * lda + gk] : T(0);
      } else {
        const int ar = row0 + tx, gk = k0 + ty;            // A element (ar, gk), stored at A[gk][ar]
        As[tx][ty] = (ar < m && gk < kend) ? A[(long long)gk * lda + ar] : T(0);
      }
      if (!tB) {
        const int gk2 = k0 + ty, bc = col0 + tx;           // B element (gk2, bc)
        Bs[ty][tx] = (bc < nn && gk2 < kend) ? B[(long long)gk2 * ldb + bc] : T(0);
      } else {
        const int gk2 = k0 + tx, bc = col0 + ty;           // B element (gk2, bc), stored at B[bc][gk2]
        Bs[tx][ty] = (bc < nn && gk2 < kend) ? B[(long long)bc * ldb + gk2] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BT; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  const bool inside = gr < m && gc < nn;
  if (splitK > 1) {
    const long long tile = ((long long)bz * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[(tile * splitK + kz) * 256 + threadIdx.x] = acc;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&count[tile], 1u) == (unsigned)(splitK - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    acc = T(0);
    for (int z = 0; z < splitK; ++z) acc += __ldcg(&part[(tile * splitK + z) * 256 + threadIdx.x]);
    if (threadIdx.x == 0) count[tile] = 0u;    // ready for the next product
  }
  if (gr < M && gc < N) C[(long long)gr * ldc + gc] = inside ? alpha * acc : T(0);
}

template <typename T>
void gemm_batched(cudaStream_t s, bool transA, bool transB, int M, int N, int K, T alpha,
                  const T* A, int lda, long long sA, const T* B, int ldb, long long sB, T beta,
                  T* C, int ldc, long long sC, int batch, const int* dynM,
                  const int* dynN, const int* dynK, const GemmScratch* scr) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  // FP64 products (C overwritten) use 16x16 tiles with a deterministic K split when the tiles
  // alone would not cover the GPU twice; the split needs the context's partial-tile scratch
  if (sizeof(T) == 8 && beta == T(0)) {
    const long long tiles = (long long)((N + 15) / 16) * ((M + 15) / 16) * batch;
    int sk = (int)((2 * 152 + tiles - 1) / tiles);
    const int maxs = (K + 15) / 16;
    if (sk > maxs) sk = maxs;
    if (!scr || !scr->part) sk = 1;
    else if (tiles * sk > GEMM_SPLIT_SLOTS) sk = (int)(GEMM_SPLIT_SLOTS / tiles);
    if (sk < 1) sk = 1;
    dim3 grid((N + 15) / 16, (M + 15) / 16, batch * sk);
    gemm_small_kernel<T><<<grid, 256, 0, s>>>(transA, transB, M, N, K, alpha, A, lda, sA, B, ldb, sB, C,
                                             ldc, sC, sk, dynM, dynN, dynK,
                                             sk > 1 ? (T*)scr->part : nullptr, sk > 1 ? scr->count : nullptr);
    return;
  }
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  gemm_kernel<T><<<grid, 256, 0, s>>>(transA, transB, M, N, K, alpha, A, lda, sA, B, ldb, sB,
                                      beta, C, ldc, sC, dynM, dynN, dynK);
}

template void gemm_batched<double>(cudaStream_t, bool, bool, int, int, int, double, const double*,
                                   int, long long, const double*, int, long long, double, double*,
                                   int, long long, int, const int*, const int*, const int*,
                                   const GemmScratch*);
template void gemm_batched<float>(cudaStream_t, bool, bool, int, int, int, float, const float*,
                                  int, long long, const float*, int, long long, float, float*,
                                  int, long long, int, const int*, const int*, const int*,
                                  const GemmScratch*);

// FP64 products in double-float arithmetic on the FP32 units (the FP32-bulk path's eigen stage):
// operands split on load as x = hi + lo (FP32 pair), each term hi_a hi_b taken exactly as its
// rounded product plus the FMA residual, the products summed with an error-free two-sum into
// (s, s_lo) and the residuals with the cross terms hi_a lo_b + lo_a hi_b in an FP32 correction;
// about 2^-44 relative to the sum of |terms|, against 2^-49 for FP64 sums of these lengths, and
// the same order as the double-float Gram matrices they multiply.  Same tiles, K split and
// deterministic partial sums as gemm_small_kernel: 16 x 16 outputs per CTA; K in chunks of 64,
// four groups of 64 threads (2 x 2 outputs each) take 16 terms of a chunk and their sums are
// added in FP64 at the end.

// x = hi + lo from the bits of x with integer operations (this GPU's FP64 pipe, conversions
// included, is a small fraction of its FP32 rate): hi keeps the sign, the exponent and the top
// 23 stored mantissa bits (truncated), lo the remaining 29 bits rounded to FP32 (x - hi exactly,
// then one rounding: |x - hi - lo| <= 2^-48 |x|).  Values below 2^-126 in magnitude become 0.
__device__ __forceinline__ float2 df_split(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  if (e < -126 || e > 127) return make_float2(0.f, 0.f);   // zero, FP32 underflow or overflow
  const unsigned sign = (unsigned)(u >> 63) << 31;
  const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((u >> 29) & 0x7FFFFFull));
  const float r = __uint2float_rn((unsigned)(u & 0x1FFFFFFFull));   // x - hi = +-r 2^(e - 52)
  const float m = (e >= -74) ? __fmul_rn(r, __uint_as_float((unsigned)(e + 75) << 23)) : ldexpf(r, e - 52);
  return make_float2(hi, sign ? -m : m);
}

constexpr int DF_KC = 64;                      // K terms of one chunk (4 groups x 16)

__global__ void __launch_bounds__(256)
gemm_df_kernel(bool tA, bool tB, int M, int N, int K, double alpha, const double* __restrict__ A, int lda,
               long long sA, const double* __restrict__ B, int ldb, long long sB, double* C, int ldc,
               long long sC, int splitK, const int* dynM, const int* dynN, const int* dynK, double* part,
               unsigned* count) {
  constexpr int BT = 16;
  __shared__ __align__(16) float2 As[DF_KC][BT], Bs[DF_KC][BT];   // (hi, lo) of A[m][k] at [k][m], B[k][n] at [k][n]
  __shared__ double red[3][BT * BT];
  __shared__ unsigned s_last;
  const int bz = blockIdx.z / splitK, kz = blockIdx.z % splitK;
  int m = M, nn = N, kk = K;
  if (dynM) m = min(m, dynM[bz]);
  if (dynN) nn = min(nn, dynN[bz]);
  if (dynK) kk = min(kk, dynK[bz]);
  const int row0 = blockIdx.y * BT, col0 = blockIdx.x * BT;
  const int tid = threadIdx.x, grp = tid >> 6, t6 = tid & 63, tx = t6 & 7, ty = t6 >> 3;
  C += bz * sC;
  if (row0 >= m || col0 >= nn) {                 // the whole tile is outside the dynamic sizes
    if (kz == 0) {
      const int gr = row0 + (tid >> 4), gc = col0 + (tid & 15);
      if (gr < M && gc < N) C[(long long)gr * ldc + gc] = 0.0;
    }
    return;
  }
  const int chunk = ((kk + splitK - 1) / splitK + BT - 1) / BT * BT;
  const int kbeg = kz * chunk, kend = min(kk, kbeg + chunk);
  A += bz * sA;
  B += bz * sB;
  float s[2][2], sl[2][2], cr[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) s[i][j] = sl[i][j] = cr[i][j] = 0.f;
  // 1024 elements of each operand per chunk, 4 per thread (positions fixed across chunks); the
  // next chunk's loads are issued before the present chunk's arithmetic
  int ka[4], ma[4], kb[4], nb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + 256 * q;
    if (!tA) { ma[q] = e >> 6; ka[q] = e & 63; } else { ka[q] = e >> 4; ma[q] = e & 15; }
    if (!tB) { kb[q] = e >> 4; nb[q] = e & 15; } else { nb[q] = e >> 6; kb[q] = e & 63; }
  }
  double xa[4], xb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ar = row0 + ma[q], gka = k0 + ka[q], bc = col0 + nb[q], gkb = k0 + kb[q];
      xa[q] = (ar < m && gka < kend) ? (tA ? A[(long long)gka * lda + ar] : A[(long long)ar * lda + gka]) : 0.0;
      xb[q] = (bc < nn && gkb < kend) ? (tB ? B[(long long)bc * ldb + gkb] : B[(long long)gkb * ldb + bc]) : 0.0;
    }
  };
  if (kbeg < kend) load(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += DF_KC) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      As[ka[q]][ma[q]] = df_split(xa[q]);
      Bs[kb[q]][nb[q]] = df_split(xb[q]);
    }
    __syncthreads();
    if (k0 + DF_KC < kend) load(k0 + DF_KC);
#pragma unroll 4
    for (int k = 16 * grp; k < 16 * grp + 16; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[k][2 * ty]);   // rows 2ty, 2ty+1: (hi, lo)
      const float4 b = *reinterpret_cast<const float4*>(&Bs[k][2 * tx]);
      const float ah[2] = {a.x, a.z}, al[2] = {a.y, a.w}, bh[2] = {b.x, b.z}, bl[2] = {b.y, b.w};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const float p = __fmul_rn(ah[i], bh[j]);
          const float e = __fmaf_rn(ah[i], bh[j], -p);
          cr[i][j] = __fmaf_rn(al[i], bh[j], __fmaf_rn(ah[i], bl[j], __fadd_rn(cr[i][j], e)));
          const float t = __fadd_rn(s[i][j], p);
          const float bp = __fsub_rn(t, s[i][j]);
          sl[i][j] = __fadd_rn(sl[i][j], __fadd_rn(__fsub_rn(s[i][j], __fsub_rn(t, bp)), __fsub_rn(p, bp)));
          s[i][j] = t;
        }
    }
    __syncthreads();
  }
  // the four groups' sums, added in FP64 in group order
  double acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      acc[i][j] = (double)s[i][j] + ((double)sl[i][j] + (double)cr[i][j]);
      if (grp > 0) red[grp - 1][(2 * ty + i) * BT + 2 * tx + j] = acc[i][j];
    }
  __syncthreads();
  if (grp > 0) return;                         // no barrier below involves the other groups
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int o = (2 * ty + i) * BT + 2 * tx + j;
      acc[i][j] = ((acc[i][j] + red[0][o]) + red[1][o]) + red[2][o];
    }
  if (splitK > 1) {
    const long long tile = ((long long)bz * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) part[(tile * splitK + kz) * 256 + (2 * ty + i) * BT + 2 * tx + j] = acc[i][j];
    __threadfence();
    asm volatile("bar.sync 1, 64;" ::: "memory");   // the 64 threads of group 0
    if (t6 == 0) s_last = (atomicAdd(&count[tile], 1u) == (unsigned)(splitK - 1));
    asm volatile("bar.sync 1, 64;" ::: "memory");
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        double v = 0.0;
        for (int z = 0; z < splitK; ++z) v += __ldcg(&part[(tile * splitK + z) * 256 + (2 * ty + i) * BT + 2 * tx + j]);
        acc[i][j] = v;
      }
    if (t6 == 0) count[tile] = 0u;             // ready for the next product
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gr = row0 + 2 * ty + i, gc = col0 + 2 * tx + j;
      if (gr < M && gc < N) C[(long long)gr * ldc + gc] = (gr < m && gc < nn) ? alpha * acc[i][j] : 0.0;
    }
}

void gemm_batched_df(cudaStream_t s, bool transA, bool transB, int M, int N, int K, const double* A, int lda,
                     long long sA, const double* B, int ldb, long long sB, double* C, int ldc, long long sC,
                     int batch, const int* dynM, const int* dynN, const int* dynK, const GemmScratch* scr) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  const long long tiles = (long long)((N + 15) / 16) * ((M + 15) / 16) * batch;
  int sk = (int)((2 * 152 + tiles - 1) / tiles);
  const int maxs = (K + 2 * DF_KC - 1) / (2 * DF_KC);     // at least two chunks per part
  if (sk > maxs) sk = maxs;
  if (!scr || !scr->part) sk = 1;
  else if (tiles * sk > GEMM_SPLIT_SLOTS) sk = (int)(GEMM_SPLIT_SLOTS / tiles);
  if (sk < 1) sk = 1;
  dim3 grid((N + 15) / 16, (M + 15) / 16, batch * sk);
  gemm_df_kernel<<<grid, 256, 0, s>>>(transA, transB, M, N, K, 1.0, A, lda, sA, B, ldb, sB, C, ldc, sC, sk, dynM,
                                     dynN, dynK, sk > 1 ? scr->part : nullptr, sk > 1 ? scr->count : nullptr);
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Seeded standard normal block Omega (Box-Muller on a counter hash).
__global__ void omega_kernel(double* Om, int n, int ks, int total) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  uint64_t h1 = splitmix64(0x1606092180000000ull + 2ull * (uint64_t)t);
  uint64_t h2 = splitmix64(0x1606092180000001ull + 2ull * (uint64_t)t);
  double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  double u2 = ((h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  Om[t] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x + 31) / 32) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// Range finder with a sparse sign embedding: X = G * Omega where every row of Omega holds
// ZETA entries +-1 in pseudo-random columns (a sparse subspace embedding; the captured energy is
// certified later by the FP64 Rayleigh quotient).  Omega is stored by column (CSR, built once per
// context): X[r][m] = sum over (i, s) in column m of s * G[r][i].  One thread per (r, m).
__global__ void __launch_bounds__(KSUB_MAX)
sparse_range_kernel(const double* __restrict__ G, const int* __restrict__ colptr,
                    const int* __restrict__ rowidx, const signed char* __restrict__ sgn, int n, int ks,
                    double* X, double* rowpart) {
  // one CTA per row r of X_l (blockDim >= ks); also the row's share of trace(G_l) and ||X_l||_F^2
  __shared__ double red[32];
  const int l = blockIdx.z, r = blockIdx.y;
  const int m = threadIdx.x;
  const double* Gr = G + ((long long)l * n + r) * n;
  double v = 0.0;
  if (m < ks) {
    for (int t = colptr[m]; t < colptr[m + 1]; ++t) v += (double)sgn[t] * Gr[rowidx[t]];
    X[((long long)l * n + r) * ks + m] = v;
  }
  const double x2 = block_sum(v * v, red);
  if (threadIdx.x == 0) {
    rowpart[2 * ((long long)l * n + r)] = Gr[r];
    rowpart[2 * ((long long)l * n + r) + 1] = x2;
  }
}

// trace(G_l) and ||X_l||_F^2 per mode from the rows' shares (one CTA per mode, fixed order)
__global__ void traces_kernel(const double* rowpart, int n, DevScalars* sc) {
  __shared__ double red[32];
  const int l = blockIdx.x;
  const double* rp = rowpart + 2ll * l * n;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += rp[2 * i];
    b += rp[2 * i + 1];
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    sc->trG[l] = a;
    sc->xnorm2[l] = b;
  }
}

// ------------------------------------------------------------------ block Gram-Schmidt
// Cooperative kernel: gridDim.x = 3 * NBC CTAs, CTA c of mode l owns rows
// [c*rows, (c+1)*rows).  The CTAs of one mode execute the same sequence of mode barriers.

// Barrier of the NBC CTAs of one mode, with a bounded wait (spins on a volatile load).  The
// kernel is launched cooperatively, so every CTA is resident and the wait normally ends after a
// few microseconds; if it does not end within ~1 s the CTA sets FLAG_TIMEOUT, stops waiting at
// this and every later barrier, and the host reports RS_ERR_TIMEOUT.  The modes are
// independent, so each has its own counter and generation.
__device__ __forceinline__ void mode_barrier(DevScalars* sc, int l, unsigned& gen, bool& poisoned) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* cnt = &sc->bar_count[32 * l];
    unsigned* gp = &sc->bar_gen[32 * l];
    __threadfence();
    unsigned arrived = atomicAdd(cnt, 1u);
    if (arrived == NBC - 1) {
      atomicExch(cnt, 0u);
      __threadfence();
      atomicAdd(gp, 1u);
    } else if (!poisoned) {
      volatile unsigned* g = gp;
      long long it = 0;
      while (*g == gen) {
        __nanosleep(32);
        if (++it > 20000000ll) {   // a second or more of polling
          atomicOr(&sc->flags, (unsigned)FLAG_TIMEOUT);
          poisoned = true;
          break;
        }
      }
    }
    __threadfence();
  }
  ++gen;
  __syncthreads();
}

// In-place lower Cholesky factor of the KB x KB matrix S (row-major, shared memory) by one
// full warp: lane i < KB holds row i of L; column jc takes jc fused multiply-adds per lane, one
// reciprocal square root and one product (FP64 issue is the cost here, so no divisions and no
// single-thread loops).  rinv[jc] = 1 / L[jc][jc].  Returns (in every lane) false if a pivot is
// not above piv_tol times its diagonal entry of S (not positive definite, or too
// ill-conditioned for Cholesky QR).
__device__ __forceinline__ bool chol8_warp(double* S, double* rinv, double piv_tol) {
  const int i = threadIdx.x & 31;
  const bool row = i < KB;
  double Lr[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) Lr[k] = 0.0;
  bool ok = true;
#pragma unroll
  for (int jc = 0; jc < KB; ++jc) {
    double v = row ? S[i * KB + jc] : 0.0;
#pragma unroll
    for (int k = 0; k < jc; ++k) v -= Lr[k] * __shfl_sync(0xffffffffu, Lr[k], jc);
    const double d = __shfl_sync(0xffffffffu, v, jc);
    const double djj = S[jc * KB + jc];
    ok = ok && (d > piv_tol * djj) && (d > 0.0);
    const double r = rsqrt(d);
    if (i == jc) Lr[jc] = d * r;
    else if (i > jc) Lr[jc] = v * r;
    if (i == 0) rinv[jc] = r;
  }
  __syncwarp();
  if (row)
#pragma unroll
    for (int k = 0; k < KB; ++k) S[i * KB + k] = (k <= i) ? Lr[k] : 0.0;
  __syncwarp();
  return ok;
}

__global__ void __launch_bounds__(256)
bcgs2_kernel(const double* __restrict__ X, double* Q, double* part, int n, int ks,
             DevScalars* sc) {
  extern __shared__ double sQ[];              // this CTA's rows of Q: (r1 - r0) x ks
  unsigned bar_gen = 0;
  bool poisoned = false;   // meaningful in thread 0 only
  const int l = blockIdx.x / NBC, c = blockIdx.x % NBC;
  const int rows = (n + NBC - 1) / NBC;
  const int r0 = min(n, c * rows), r1 = min(n, r0 + rows);
  const int nr = r1 - r0;
  const double* Xl = X + (long long)l * n * ks;
  double* Ql = Q + (long long)l * n * ks;
  // part layout: [2][3][NBC][ks*KB + KB*KB].  Partials written by other SMs are read with
  // __ldcg (L2, bypassing the non-coherent L1) after the grid barrier.
  const long long pstride = (long long)ks * KB + KB * KB;
  auto pbuf = [&](int phase, int mode, int cta) {
    return part + (((long long)(phase & 1) * 3 + mode) * NBC + cta) * pstride;
  };
  // reduced sums of a phase: [2][3][pstride] after the partials
  auto fbuf = [&](int phase, int mode) {
    return part + (2ll * 3 * NBC + (long long)(phase & 1) * 3 + mode) * pstride;
  };
  __shared__ double h[KSUB_MAX * KB];
  __shared__ double S[KB * KB];
  __shared__ double rinv[KB];
  __shared__ double red[256];                 // split FP64 sums (blockDim.x = 256)
  __shared__ int s_stop;
  const double xn2 = sc->xnorm2[l];
  const double guard2 = 1e6 * 4.93e-32 * xn2;   // (1e3 * 2.22e-16)^2 * ||X||^2
  int kq = 0;
  bool stop = !(xn2 > 0.0);
  bool fallback = false;
  if (stop && c == 0 && threadIdx.x == 0) atomicOr(&sc->stopmask, 1u << l);
  int phase = 0;
  const int tid = threadIdx.x;
  auto sq = [&](int ii, int col) -> double& { return sQ[ii * ks + col]; };   // ii = i - r0
  auto gq = [&](int i, int col) { return __ldcg(Ql + (long long)i * ks + col); };

  for (int e = tid; e < nr * ks; e += blockDim.x) sQ[e] = 0.0;
  __syncthreads();

  // per-row helpers on the working block B = Q[:, kq:kq+KB] (own rows, shared memory)
  auto partial_h = [&](double* P) {           // P[a*KB+jc] = sum_{own rows} Q[i][a] B[i][jc]
    for (int e = tid; e < kq * KB; e += blockDim.x) {
      int a = e / KB, jc = e % KB;
      double v = 0.0;
      for (int ii = 0; ii < nr; ++ii) v += sq(ii, a) * sq(ii, kq + jc);
      P[e] = v;
    }
  };
  auto partial_S = [&](double* P) {           // P[a*KB+b] = sum_{own rows} B[i][a] B[i][b]
    for (int e = tid; e < KB * KB; e += blockDim.x) {
      int a = e / KB, b = e % KB;
      double v = 0.0;
      for (int ii = 0; ii < nr; ++ii) v += sq(ii, kq + a) * sq(ii, kq + b);
      P[e] = v;
    }
  };
  // dst[e] = sum over the mode's CTAs of their partial e (offset off in the phase buffer) for
  // e in [eb, ee): 8 lanes per output, lane r adds the partials of CTAs r, r + 8, ...
  // (independent loads, four outputs in flight per lane), then a fixed xor tree over the 8 lanes
  auto reduce_partials = [&](int ph, long long off, int eb, int ee, double* dst) {
    const int g = tid >> 3, r = tid & 7, ng = (int)blockDim.x >> 3;
    for (int e0 = eb; e0 < ee; e0 += 4 * ng) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * ng + g;
        v[u] = 0.0;
        if (e < ee) {
#pragma unroll
          for (int t = 0; t < NBC / 8; ++t) v[u] += __ldcg(pbuf(ph, l, r + 8 * t) + off + e);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        double w = v[u];
        w += __shfl_xor_sync(0xffffffffu, w, 4);
        w += __shfl_xor_sync(0xffffffffu, w, 2);
        w += __shfl_xor_sync(0xffffffffu, w, 1);
        const int e = e0 + u * ng + g;
        if (e < ee && r == 0) dst[e] = w;
      }
    }
  };
  // CTA c sums its slice of the E outputs at offset off and publishes them in the phase's
  // final buffer (read by every CTA of the mode after the next barrier): each sum is formed
  // once instead of in every CTA
  auto reduce_slice = [&](int ph, long long off, int E) {
    const int per = (E + NBC - 1) / NBC;
    const int eb = min(E, c * per), ee = min(E, eb + per);
    reduce_partials(ph, off, eb, ee, fbuf(ph, l) + off);
  };
  auto fetch = [&](int ph, long long off, int E, double* dst) {
    for (int e = tid; e < E; e += blockDim.x) dst[e] = __ldcg(fbuf(ph, l) + off + e);
  };
  auto reduce_S = [&](int ph, int off) { reduce_partials(ph, off, 0, KB * KB, S); };
  // B -= Q[:, :kq] h on own rows; each output's sum over a is split over P threads
  auto subtract_Qh = [&]() {
    const int no = nr * KB;
    if (no == 0) return;
    const int P = max(1, min(4, (int)blockDim.x / no));
    if (tid < P * no) {
      const int o = tid % no, q = tid / no;
      const int ii = o / KB, jc = o % KB;
      double v = 0.0;
      for (int a = q; a < kq; a += P) v += sq(ii, a) * h[a * KB + jc];
      red[tid] = v;
    }
    __syncthreads();
    if (tid < no) {
      double acc = red[tid];
      for (int q = 1; q < P; ++q) acc += red[q * no + tid];
      sq(tid / KB, kq + tid % KB) -= acc;
    }
    __syncthreads();
  };
  // S -= h^T h (the Gram of the reprojected block); each entry's sum over m split over 4 threads
  auto subtract_hth = [&]() {
    {
      const int o = tid & (KB * KB - 1), q = tid >> 6;
      const int a = o / KB, b = o % KB;
      double v = 0.0;
      for (int m = q; m < kq; m += 4) v += h[m * KB + a] * h[m * KB + b];
      red[tid] = v;
    }
    __syncthreads();
    if (tid < KB * KB) S[tid] -= ((red[tid] + red[64 + tid]) + red[128 + tid]) + red[192 + tid];
    __syncthreads();
  };
  auto solve_LT = [&]() {                     // B <- B L^{-T} on own rows (L in S, 1/diag in rinv)
    for (int ii = tid; ii < nr; ii += blockDim.x) {
      double y[KB];
      for (int jc = 0; jc < KB; ++jc) {
        double v = sq(ii, kq + jc);
        for (int k = 0; k < jc; ++k) v -= S[jc * KB + k] * y[k];
        y[jc] = v * rinv[jc];
      }
      for (int jc = 0; jc < KB; ++jc) sq(ii, kq + jc) = y[jc];
    }
  };
  auto block_to_global = [&]() {              // own rows of the working block -> Q
    for (int e = tid; e < nr * KB; e += blockDim.x) {
      int ii = e / KB, jc = e % KB;
      Ql[(long long)(r0 + ii) * ks + kq + jc] = sq(ii, kq + jc);
    }
  };
  auto block_from_global = [&]() {            // Q -> own rows of the working block
    for (int e = tid; e < nr * KB; e += blockDim.x) {
      int ii = e / KB, jc = e % KB;
      if (kq + jc < ks) sq(ii, kq + jc) = gq(r0 + ii, kq + jc);
    }
  };
  // Fallback for a block too ill-conditioned for Cholesky QR (fast-decaying spectra): CTA 0
  // of the mode orthonormalises the 8 columns one by one in global memory (classical
  // Gram-Schmidt, two passes, against the block's accepted columns; the two projections
  // against the earlier blocks were already done in parallel), drops columns that fall below
  // the noise guard, compacts the accepted ones to the front and publishes their count.
  __shared__ double fred[8][KB];
  __shared__ double fd[KB];
  __shared__ int s_acc;
  auto row = [&](int i) { return Ql + (long long)i * ks; };
  auto fallback_block = [&]() {
    if (tid == 0) s_acc = 0;
    __syncthreads();
    for (int jc = 0; jc < KB; ++jc) {
      const int acc = s_acc;
      for (int pass = 0; pass < 2 && acc > 0; ++pass) {
        double d[KB];
        for (int a = 0; a < KB; ++a) d[a] = 0.0;
        for (int i = tid; i < n; i += blockDim.x) {
          double v = gq(i, kq + jc);
          for (int a = 0; a < acc; ++a) d[a] += gq(i, kq + a) * v;
        }
        for (int a = 0; a < acc; ++a) {
          double v = d[a];
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
          if ((tid & 31) == 0) fred[tid >> 5][a] = v;
        }
        __syncthreads();
        if (tid < acc) {
          double v = 0.0;
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += fred[w][tid];
          fd[tid] = v;
        }
        __syncthreads();
        for (int i = tid; i < n; i += blockDim.x) {
          double v = gq(i, kq + jc);
          for (int a = 0; a < acc; ++a) v -= fd[a] * gq(i, kq + a);
          row(i)[kq + jc] = v;
        }
        __syncthreads();
      }
      double nv = 0.0;
      for (int i = tid; i < n; i += blockDim.x) { double v = gq(i, kq + jc); nv += v * v; }
      for (int o = 16; o > 0; o >>= 1) nv += __shfl_down_sync(0xffffffffu, nv, o);
      if ((tid & 31) == 0) fred[tid >> 5][0] = nv;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += fred[w][0];
        fd[0] = t;
      }
      __syncthreads();
      const double nv2 = fd[0];
      if (nv2 >= guard2 && nv2 > 0.0) {
        const double sc1 = 1.0 / sqrt(nv2);
        for (int i = tid; i < n; i += blockDim.x) row(i)[kq + acc] = gq(i, kq + jc) * sc1;
        __syncthreads();
        if (tid == 0) s_acc = acc + 1;
      }
      __syncthreads();
    }
    const int acc = s_acc;
    for (int e = tid; e < n * (KB - acc); e += blockDim.x) {
      int i = e / (KB - acc), jc = acc + e % (KB - acc);
      row(i)[kq + jc] = 0.0;
    }
    if (tid == 0) sc->blk_acc[l] = acc;
  };

  auto mark_stop = [&](unsigned flag) {
    stop = true;
    if (c == 0 && tid == 0) {
      atomicOr(&sc->stopmask, 1u << l);
      if (flag) atomicOr(&sc->flags, flag);
    }
  };

  for (int s = 0; s < ks; s += KB) {
    if (stop) break;                          // the same decision in every CTA of the mode
    if (!stop)
      for (int e = tid; e < nr * KB; e += blockDim.x) {
        int ii = e / KB, jc = e % KB;
        sq(ii, kq + jc) = Xl[(long long)(r0 + ii) * ks + s + jc];
      }
    __syncthreads();   // the partial products below read rows written by other threads
    // (A) first projection against the accepted columns
    if (kq > 0) {
      partial_h(pbuf(phase, l, c));
      mode_barrier(sc, l, bar_gen, poisoned);
      reduce_slice(phase, 0, kq * KB);
      mode_barrier(sc, l, bar_gen, poisoned);
      fetch(phase, 0, kq * KB, h);
      __syncthreads();
      subtract_Qh();
    }
    ++phase;
    // (B) second projection and (C) the Gram of the block from one reduction, as in (D):
    //     h = Q^T B, S = B^T B, B <- B - Q h, S <- S - h^T h (after (A) h is small, so the
    //     difference loses nothing); then the norm test and the first Cholesky QR.  Without
    //     accepted columns S alone, summed by every CTA after one barrier.
    if (kq > 0) {
      double* P = pbuf(phase, l, c);
      partial_h(P);
      partial_S(P + (long long)ks * KB);
      mode_barrier(sc, l, bar_gen, poisoned);
      reduce_slice(phase, 0, kq * KB);
      reduce_slice(phase, (long long)ks * KB, KB * KB);
      mode_barrier(sc, l, bar_gen, poisoned);
      fetch(phase, 0, kq * KB, h);
      fetch(phase, (long long)ks * KB, KB * KB, S);
      __syncthreads();
      subtract_hth();
      subtract_Qh();
    } else {
      partial_S(pbuf(phase, l, c));
      mode_barrier(sc, l, bar_gen, poisoned);
      reduce_S(phase, 0);
    }
    block_to_global();                       // CTA 0 reads every row if the block falls back
    {
      __syncthreads();
      if (tid < 32) {
        double tr = 0.0;
        for (int a = 0; a < KB; ++a) tr += S[a * KB + a];
        const bool tiny = tr < guard2;
        const bool ok = tiny ? false : chol8_warp(S, rinv, 1e-10);
        if (tid == 0) s_stop = tiny ? 1 : (ok ? 0 : 3);
      }
      __syncthreads();
      if (s_stop == 1) mark_stop(0u);
      else if (s_stop == 3) {
        fallback = true;
        // the same decision in every CTA of the mode: one more barrier, so that CTA 0 sees every
        // CTA's rows of the block in global memory
        mode_barrier(sc, l, bar_gen, poisoned);
        if (c == 0) {
          if (tid == 0) atomicAdd(&sc->fallbacks, 1);
          fallback_block();
        }
      }
      else solve_LT();
    }
    __syncthreads();
    ++phase;
    // (D) reprojection and second Cholesky QR from one reduction:
    //     h = Q^T B, S = B^T B, (B - Q h)^T (B - Q h) = S - h^T h
    if (!stop && !fallback) {
      double* P = pbuf(phase, l, c);
      if (kq > 0) partial_h(P);
      partial_S(P + (long long)ks * KB);
    }
    mode_barrier(sc, l, bar_gen, poisoned);
    if (!stop && !fallback) {
      if (kq > 0) reduce_slice(phase, 0, kq * KB);
      reduce_slice(phase, (long long)ks * KB, KB * KB);
    }
    mode_barrier(sc, l, bar_gen, poisoned);
    if (!stop && !fallback) {
      if (kq > 0) fetch(phase, 0, kq * KB, h);
      fetch(phase, (long long)ks * KB, KB * KB, S);
      __syncthreads();
      if (kq > 0) {
        subtract_hth();
        subtract_Qh();
      }
      if (tid < 32) {
        const bool ok = chol8_warp(S, rinv, 0.0);
        if (tid == 0) s_stop = ok ? 0 : 2;
      }
      __syncthreads();
      if (s_stop) mark_stop((unsigned)FLAG_CHOL);
      else solve_LT();
    }
    __syncthreads();
    ++phase;
    if (!stop && fallback) {
      block_from_global();                   // the block as CTA 0 left it
      const int acc = (int)__ldcg(&sc->blk_acc[l]);
      kq += acc;
      fallback = false;
      if (acc == 0) mark_stop(0u);
      if (kq + KB > ks && !stop) mark_stop(0u);
    } else if (!stop) {
      kq += KB;
      if (kq + KB > ks) mark_stop(0u);
    } else {
      for (int e = tid; e < nr * KB; e += blockDim.x) {
        int ii = e / KB, jc = e % KB;
        if (kq + jc < ks) sq(ii, kq + jc) = 0.0;
      }
    }
    __syncthreads();
  }
  // own rows back to Q
  for (int e = tid; e < nr * ks; e += blockDim.x) Ql[(long long)r0 * ks + e] = sQ[e];
  if (c == 0 && tid == 0) sc->k_eff[l] = kq;
}

// ------------------------------------------------------------------ FP32 Jacobi
// One CTA per mode: A (ke x ke, FP32, scaled by 1/max diag) in shared memory, V accumulated.
// Parallel (round-robin) ordering: each round applies ke/2 disjoint rotations.
__global__ void __launch_bounds__(1024)
jacobi32_kernel(const double* __restrict__ Tm, double* Wm, int ks, DevScalars* sc, int max_sweeps,
                float tol) {
  extern __shared__ float smem[];
  const int l = blockIdx.x;
  const int ke0 = sc->k_eff[l];
  const int ke = (ke0 + 1) & ~1;               // even size (padding row/column is zero)
  const int ld = ke + 1;
  float* A = smem;                              // ke x ld
  float* V = smem + ke * ld;                    // ke x ld
  __shared__ float cs[KSUB_MAX / 2], sn[KSUB_MAX / 2], dpp[KSUB_MAX / 2], dqq[KSUB_MAX / 2];
  __shared__ int pp[KSUB_MAX / 2], qq[KSUB_MAX / 2];
  __shared__ int s_rot;
  __shared__ double s_scale;
  const double* T = Tm + (long long)l * ks * ks;
  double* W = Wm + (long long)l * ks * ks;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < ke0; ++i) m = fmax(m, fabs(T[(long long)i * ks + i]));
    s_scale = (m > 0.0) ? 1.0 / m : 1.0;
  }
  __syncthreads();
  const double scl = s_scale;
  for (int e = tid; e < ke * ke; e += nt) {
    int i = e / ke, jc = e % ke;
    double v = (i < ke0 && jc < ke0) ? T[(long long)i * ks + jc] * scl : 0.0;
    A[i * ld + jc] = (float)v;
    V[i * ld + jc] = (i == jc) ? 1.f : 0.f;
  }
  __syncthreads();
  const int half = ke / 2;
  // round-robin pairing (position 0 fixed, the others rotate): pair m of round r is
  // (a, b) = (m ? 1 + (m - 1 + r) mod (ke - 1) : 0, 1 + (ke - 2 - m + r) mod (ke - 1)); thread m
  // keeps its pair in registers and advances it by one position per round (the integer
  // divisions of the closed form had been the larger part of the parameter phase)
  int ra = 0, rb = 0;
  if (tid < half) {
    ra = tid;
    rb = (tid == 0) ? ke - 1 : ke - 1 - tid;
  }
  for (int sweep = 0; sweep < max_sweeps && ke > 1; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < ke - 1; ++round) {
      for (int m = tid; m < half; m += nt) {        // half <= KSUB_MAX / 2 < nt: one pair per thread
        const int a = ra, b = rb;
        int p = min(a, b), q = max(a, b);
        pp[m] = p;
        qq[m] = q;
        float apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
        float c = 1.f, s = 0.f, t = 0.f;
        // this phase runs on one warp while the others wait: fast division and reciprocal
        // square root (about 2 ulp) instead of IEEE division and square root; the
        // rotation stays orthogonal (c = 1/sqrt(1 + t^2), s = t c) and the diagonal update below
        // uses the t that is applied
        if (apq != 0.f && apq * apq > tol * tol * fabsf(app * aqq)) {
          const float theta = __fdividef(aqq - app, 2.f * apq);
          const float w = fmaf(theta, theta, 1.f);
          t = copysignf(__fdividef(1.f, fabsf(theta) + w * rsqrtf(w)), theta);
          c = rsqrtf(fmaf(t, t, 1.f));
          s = t * c;
          s_rot = 1;
        }
        cs[m] = c;
        sn[m] = s;
        dpp[m] = app - t * apq;     // graded-accurate diagonal of the rotated pair
        dqq[m] = aqq + t * apq;
      }
      if (tid < half) {                             // the pairs of the next round
        if (tid != 0) ra = (ra == ke - 1) ? 1 : ra + 1;
        rb = (rb == ke - 1) ? 1 : rb + 1;
      }
      __syncthreads();
      // rows: A[p,:], A[q,:] -- warp w takes pairs w, w + 8, ..., lanes take columns
      for (int m = warp; m < half; m += nwarp) {
        const float s = sn[m];
        if (s == 0.f) continue;
        const int p = pp[m], q = qq[m];
        const float c = cs[m];
        float* Ap = A + p * ld;
        float* Aq = A + q * ld;
        for (int col = lane; col < ke; col += 32) {
          float ap = Ap[col], aq = Aq[col];
          Ap[col] = c * ap - s * aq;
          Aq[col] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // columns: A[:,p], A[:,q] and V[:,p], V[:,q]; the 2x2 block of each rotated pair takes
      // its exact values (graded-accurate diagonal, zero off-diagonal)
      for (int m = warp; m < half; m += nwarp) {
        const float s = sn[m];
        if (s == 0.f) continue;
        const int p = pp[m], q = qq[m];
        const float c = cs[m];
        for (int row = lane; row < ke; row += 32) {
          float* Vr = V + row * ld;
          float vp = Vr[p], vq = Vr[q];
          Vr[p] = c * vp - s * vq;
          Vr[q] = s * vp + c * vq;
          float* Ar = A + row * ld;
          if (row == p) {
            Ar[p] = dpp[m];
            Ar[q] = 0.f;
          } else if (row == q) {
            Ar[q] = dqq[m];
            Ar[p] = 0.f;
          } else {
            float ap = Ar[p], aq = Ar[q];
            Ar[p] = c * ap - s * aq;
            Ar[q] = s * ap + c * aq;
          }
        }
      }
      __syncthreads();
    }
    if (tid == 0) atomicAdd(&sc->jacobi_sweeps, 1);
    if (s_rot == 0) break;
    __syncthreads();
  }
  // W (ks x ks, FP64): eigenvectors in the leading ke0 x ke0 block, zero elsewhere
  for (long long e = tid; e < (long long)ks * ks; e += nt) {
    int i = (int)(e / ks), jc = (int)(e % ks);
    W[e] = (i < ke0 && jc < ke0) ? (double)V[i * ld + jc] : 0.0;
  }
}

// The same Jacobi pass with one barrier per round (subspaces up to JF_KMAX).  A is kept in slot
// order: with the round-robin schedule, pair m of every round is slots (m, ke-1-m), and between
// rounds the indices move one slot down (slot 1 wraps to ke-1, slot 0 stays), so round r reads
// A_r in its slot order and writes A_{r+1} = J_r^T A_r J_r straight into the next round's slot
// order (the other copy).  Thread (warp w, lane i) owns the 2 x 2 blocks of pairs (w + 32 u,
// i + 32 v): the slots of a block never change, so its addresses and whether one of its entries
// becomes the off-diagonal of a pair of the next round are fixed; that entry gives the pair's
// rotation at once (its diagonal is the rotated diagonal of round r), so rotations, A and V
// never wait for one another within a round.  V stays in the original index order: the two
// indices of a pair in round r are closed-form and each thread follows its own pairs.
constexpr int JF_KMAX = 128;
constexpr int JF_THREADS = 1024;

__device__ __forceinline__ float jf_rot(float a, float b, float c, float s, int i) {
  return i ? __fmaf_rn(s, a, __fmul_rn(c, b)) : __fmaf_rn(c, a, -__fmul_rn(s, b));
}

struct JfShared {
  float2 rot[2][JF_KMAX / 2];                  // (c, s) of pair m
  float dsl[2][JF_KMAX];                       // diagonal of each slot after the round's rotation
  int s_cnt[32];                               // rotations of each sweep (nonzero flag)
};

// rotation of pair m (slots m, ke-1-m) for the round in buffer b and sweep sw
__device__ __forceinline__ void jf_set_rotation(JfShared& S, int ke, float tol, int b, int sw, int m, float apq,
                                                float app, float aqq) {
  float c = 1.f, s = 0.f, t = 0.f;
  if (apq != 0.f && apq * apq > tol * tol * fabsf(app * aqq)) {
    const float theta = __fdividef(aqq - app, 2.f * apq);
    const float w = fmaf(theta, theta, 1.f);
    t = copysignf(__fdividef(1.f, fabsf(theta) + w * rsqrtf(w)), theta);
    c = rsqrtf(fmaf(t, t, 1.f));
    s = t * c;
    S.s_cnt[sw] = 1;
  }
  S.rot[b][m] = make_float2(c, s);
  S.dsl[b][m] = app - t * apq;                 // graded-accurate diagonal of the rotated pair
  S.dsl[b][ke - 1 - m] = aqq + t * apq;
}

__device__ __forceinline__ int jf_snext(int k, int ke) { return k == 0 ? 0 : (k == 1 ? ke - 1 : k - 1); }

// the rounds of the pass; B x B blocks and B V pairs per thread (ke <= 64 B)
template <int B>
__device__ void jf_rounds(float* A0, float* A1, float* V, int ke, int ld, int sweeps, float tol, JfShared& S,
                          DevScalars* sc) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = ke / 2, rounds = ke - 1;
  // fixed per block: read offsets (slots s/t of pair m1) x (slots s/t of pair m2), write offsets
  // in the next slot order, and the entry on the next round's anti-diagonal (-1: none; only in
  // blocks m1 < m2, which hold at most one)
  int rd[B * B][4], wr[B * B][4], anti[B * B], tgt[B * B], dp[B * B], dq[B * B];
#pragma unroll
  for (int u = 0; u < B * B; ++u) {
    const int m1 = warp + 32 * (u / B), m2 = lane + 32 * (u % B);
    const int sl[2] = {m1, ke - 1 - m1}, cl[2] = {m2, ke - 1 - m2};
    anti[u] = -1;
    tgt[u] = dp[u] = dq[u] = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = sl[e >> 1], c = cl[e & 1];
      const int rn = jf_snext(r, ke), cn = jf_snext(c, ke);
      rd[u][e] = r * ld + c;
      wr[u][e] = rn * ld + cn;
      if (m1 < m2 && m2 < half && rn + cn == ke - 1) {
        anti[u] = e;
        tgt[u] = min(rn, cn);
        dp[u] = rn < cn ? r : c;                 // slot (round r) of the pair's first index
        dq[u] = rn < cn ? c : r;
      }
    }
  }
  int pa[B], pb[B];
#pragma unroll
  for (int u = 0; u < B; ++u) {
    pa[u] = warp + 32 * u;
    pb[u] = ke - 1 - (warp + 32 * u);
  }
  int sw = 0, j = 0;                             // sweep and round within it
  for (int R = 0; sw < sweeps; ++R) {
    const int b = R & 1;
    const float* A = b ? A1 : A0;
    float* An = b ? A0 : A1;
    const int swn = (j + 1 == rounds) ? sw + 1 : sw;
    const bool more = swn < sweeps;
#pragma unroll
    for (int u = 0; u < B * B; ++u) {
      const int m1 = warp + 32 * (u / B), m2 = lane + 32 * (u % B);
      if (m1 < half && m2 < half) {
        if (m1 == m2) {
          const int s1 = m1, t1 = ke - 1 - m1;
          const float d0 = S.dsl[b][s1], d1 = S.dsl[b][t1];
          An[wr[u][0]] = d0;
          An[wr[u][1]] = 0.f;
          An[wr[u][2]] = 0.f;
          An[wr[u][3]] = d1;
          if (more && ke == 2) jf_set_rotation(S, ke, tol, b ^ 1, swn, 0, 0.f, d0, d1);   // the same pair
        } else {
          const float2 r1 = S.rot[b][m1], r2 = S.rot[b][m2];
          const float x00 = A[rd[u][0]], x01 = A[rd[u][1]], x10 = A[rd[u][2]], x11 = A[rd[u][3]];
          const float u0 = jf_rot(x00, x10, r1.x, r1.y, 0), u1 = jf_rot(x01, x11, r1.x, r1.y, 0);
          const float w0 = jf_rot(x00, x10, r1.x, r1.y, 1), w1 = jf_rot(x01, x11, r1.x, r1.y, 1);
          const float y00 = jf_rot(u0, u1, r2.x, r2.y, 0), y01 = jf_rot(u0, u1, r2.x, r2.y, 1);
          const float y10 = jf_rot(w0, w1, r2.x, r2.y, 0), y11 = jf_rot(w0, w1, r2.x, r2.y, 1);
          An[wr[u][0]] = y00;
          An[wr[u][1]] = y01;
          An[wr[u][2]] = y10;
          An[wr[u][3]] = y11;
          const int e = anti[u];
          if (more && e >= 0) {
            const float y = e == 0 ? y00 : (e == 1 ? y01 : (e == 2 ? y10 : y11));
            jf_set_rotation(S, ke, tol, b ^ 1, swn, tgt[u], y, S.dsl[b][dp[u]], S.dsl[b][dq[u]]);
          }
        }
      }
    }
    // V <- V J_r: columns (index at slot m, index at slot ke-1-m) of each pair
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int m = warp + 32 * u;
      if (m < half) {
        const float2 r = S.rot[b][m];
        if (r.y != 0.f) {
          const int p = pa[u], q = pb[u];
#pragma unroll
          for (int k = 0; k < 2 * B; ++k) {
            const int row = lane + 32 * k;
            if (row < ke) {
              float* Vr = V + row * ld;
              const float vp = Vr[p], vq = Vr[q];
              Vr[p] = r.x * vp - r.y * vq;
              Vr[q] = r.y * vp + r.x * vq;
            }
          }
        }
        if (m != 0) pa[u] = (pa[u] == ke - 1) ? 1 : pa[u] + 1;
        pb[u] = (pb[u] == ke - 1) ? 1 : pb[u] + 1;
      }
    }
    __syncthreads();
    if (++j == rounds) {                         // end of a sweep
      if (tid == 0) atomicAdd(&sc->jacobi_sweeps, 1);
      if (S.s_cnt[sw] == 0) break;               // no rotation in this sweep
      j = 0;
      ++sw;
      // the next sweep rotates nothing unless a pair of the present A meets the rotation test
      // (nothing changes before that pair's round): test all pairs at once
      if (sw < sweeps) {
        int any = 0;
        for (int e = tid; e < ke * ke; e += blockDim.x) {
          const int r = e / ke, c = e - (e / ke) * ke;
          if (r < c) {
            const float apq = An[r * ld + c];
            if (apq != 0.f && apq * apq > tol * tol * fabsf(An[r * ld + r] * An[c * ld + c])) any = 1;
          }
        }
        if (__syncthreads_or(any) == 0) break;
      }
    }
  }
}

__global__ void __launch_bounds__(JF_THREADS)
jacobi32f_kernel(const double* __restrict__ Tm, double* Wm, int ks, DevScalars* sc, int max_sweeps,
                 float tol) {
  extern __shared__ float smem[];
  __shared__ JfShared S;
  __shared__ double s_scale;
  const int l = blockIdx.x;
  const int ke0 = sc->k_eff[l];
  const int ke = (ke0 + 1) & ~1;               // even size (padding row/column is zero)
  const int ld = ke + 1;
  float* const A0 = smem;                      // A_r and A_{r+1} in slot order, alternating
  float* const A1 = smem + ke * ld;
  float* const V = smem + 2 * ke * ld;         // original index order
  const double* T = Tm + (long long)l * ks * ks;
  double* W = Wm + (long long)l * ks * ks;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < 32) {                              // largest diagonal entry (one warp)
    double m = 0.0;
    for (int i = tid; i < ke0; i += 32) m = fmax(m, fabs(T[(long long)i * ks + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (tid == 0) s_scale = (m > 0.0) ? 1.0 / m : 1.0;
    S.s_cnt[tid] = 0;
  }
  __syncthreads();
  const double scl = s_scale;
  for (int e = tid; e < ke * ke; e += nt) {
    const int i = e / ke, jc = e % ke;
    const double v = (i < ke0 && jc < ke0) ? T[(long long)i * ks + jc] * scl : 0.0;
    A0[i * ld + jc] = (float)v;                // round 0: slot k holds index k
    V[i * ld + jc] = (i == jc) ? 1.f : 0.f;
  }
  const int half = ke / 2;
  const int sweeps = min(max_sweeps, 31);
  __syncthreads();
  if (ke > 1 && sweeps > 0) {
    for (int m = tid; m < half; m += nt)
      jf_set_rotation(S, ke, tol, 0, 0, m, A0[m * ld + (ke - 1 - m)], A0[m * ld + m],
                      A0[(ke - 1 - m) * ld + (ke - 1 - m)]);
    __syncthreads();
    if (ke <= 64)
      jf_rounds<1>(A0, A1, V, ke, ld, sweeps, tol, S, sc);
    else
      jf_rounds<2>(A0, A1, V, ke, ld, sweeps, tol, S, sc);
  }
  // W (ks x ks, FP64): eigenvectors in the leading ke0 x ke0 block, zero elsewhere
  for (long long e = tid; e < (long long)ks * ks; e += nt) {
    const int i = (int)(e / ks), jc = (int)(e % ks);
    W[e] = (i < ke0 && jc < ke0) ? (double)V[i * ld + jc] : 0.0;
  }
}

// M = I - E/2 + 3/8 E^2 (Newton-Schulz step for (Q^T Q)^{-1/2}) from E = Q^T Q - I and
// E2 = E^2 on the leading ke block; zero elsewhere.  In place on E is allowed.
__global__ void ns_matrix_kernel(const double* E, const double* E2, double* M, int ks,
                                 const DevScalars* sc) {
  int l = blockIdx.y;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ks * ks) return;
  int i = e / ks, jc = e % ks;
  int ke = sc->k_eff[l];
  long long o = (long long)l * ks * ks + e;
  double v = 0.0;
  if (i < ke && jc < ke) v = (i == jc ? 1.0 : 0.0) - 0.5 * E[o] + 0.375 * E2[o];
  M[o] = v;
}

// E = Q^T Q - I in place (leading ke block only; zero outside)
__global__ void sub_identity_kernel(double* A, int ks, const DevScalars* sc) {
  int l = blockIdx.y;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ks * ks) return;
  int i = e / ks, jc = e % ks;
  int ke = sc->k_eff[l];
  long long o = (long long)l * ks * ks + e;
  A[o] = (i < ke && jc < ke) ? A[o] - (i == jc ? 1.0 : 0.0) : 0.0;
}

// ------------------------------------------------------------------ rank selection
// One CTA per mode: sort diag(T) descending, tail(r) = (trG - trT) + sum_{i>=r} lambda_i,
// r = min{r >= 1 : tail(r) <= eps^2/3 * trG}, bounded by rank_cap and rmax.
__global__ void rank_select_kernel(const double* Tm, int ks, double eps, int cap, int rmax,
                                   int* order, double* ev, DevScalars* sc) {
  const int l = blockIdx.x;
  const int ke = sc->k_eff[l];
  const double* T = Tm + (long long)l * ks * ks;
  __shared__ double d[KSUB_MAX];
  __shared__ int ord[KSUB_MAX];
  for (int i = threadIdx.x; i < ke; i += blockDim.x) d[i] = T[(long long)i * ks + i];
  __syncthreads();
  // rank sort (ties broken by index)
  for (int i = threadIdx.x; i < ke; i += blockDim.x) {
    int pos = 0;
    for (int jc = 0; jc < ke; ++jc)
      if (d[jc] > d[i] || (d[jc] == d[i] && jc < i)) ++pos;
    ord[pos] = i;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ks; i += blockDim.x) {
    order[l * ks + i] = (i < ke) ? ord[i] : -1;
    ev[l * ks + i] = (i < ke) ? d[ord[i]] : 0.0;
  }
  if (threadIdx.x == 0) {
    double trG = sc->trG[l];
    double trT = 0.0;
    for (int i = 0; i < ke; ++i) trT += d[i];
    sc->trT[l] = trT;
    int r = 0;
    double tail_r = 0.0;
    if (trG > 0.0 && ke > 0) {
      double outside = fmax(trG - trT, 0.0);
      double budget = eps * eps / 3.0 * trG;
      // tail(r) for r = ke .. 1
      double tail = outside;
      int found = -1;
      double tail_found = 0.0;
      for (int rr = ke; rr >= 1; --rr) {
        // tail currently = tail(rr)
        if (tail <= budget) { found = rr; tail_found = tail; }
        else break;
        tail += fmax(d[ord[rr - 1]], 0.0);
      }
      bool capped = false;
      if (found < 0) { found = ke; tail_found = outside; capped = true; }
      r = found;
      int lim = rmax;
      if (cap > 0 && cap < lim) lim = cap;
      if (r > lim) {
        capped = true;
        double t2 = outside;
        for (int i = lim; i < ke; ++i) t2 += fmax(d[ord[i]], 0.0);
        r = lim;
        tail_found = t2;
      }
      tail_r = tail_found / trG;
      if (capped) atomicOr(&sc->flags, (unsigned)FLAG_RANK_CAPPED);
    }
    sc->rank[l] = r;
    sc->tail_rel[l] = tail_r;
  }
}

// Z[l][i][a] = Q[l][i][order[a]] for a < r_l, 0 otherwise (FP64 and FP32 copies)
__global__ void gather_Z_kernel(const double* Q, const int* order, int n, int ks, int rmax,
                                const DevScalars* sc, double* Z64, float* Z32) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tot = 3ll * n * rmax;
  if (e >= tot) return;
  int l = (int)(e / ((long long)n * rmax));
  int rem = (int)(e % ((long long)n * rmax));
  int i = rem / rmax, a = rem % rmax;
  double v = 0.0;
  if (a < sc->rank[l]) v = Q[((long long)l * n + i) * ks + order[l * ks + a]];
  Z64[e] = v;
  Z32[e] = (float)v;
}

// ------------------------------------------------------------------ driver
// sweeps and relative off-diagonal tolerance of the Jacobi pass
constexpr int JACOBI_SWEEPS = 16;
constexpr float JACOBI_TOL = 1e-5f;
// T <- W^T T W for the leading ke block (two k x k products through T2k)
// The eigen stage's FP64 products: double-float on the FP32-bulk path, FP64 on the FP64 path
// (C = op(A) op(B), overwritten; deterministic K split through the context's scratch)
static void eig_prod(Ctx& c, bool tA, bool tB, int M, int N, int K, const double* A, int lda, long long sA,
                     const double* B, int ldb, long long sB, double* C, int ldc, long long sC, int batch,
                     const int* dM, const int* dN, const int* dK) {
  if (c.fp64)
    gemm_batched<double>(c.stream, tA, tB, M, N, K, 1.0, A, lda, sA, B, ldb, sB, 0.0, C, ldc, sC, batch, dM, dN, dK,
                         &c.gscr);
  else
    gemm_batched_df(c.stream, tA, tB, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, dM, dN, dK, &c.gscr);
}

static void congruence(Ctx& c, double* Tm, const double* Wm) {
  const int ks = c.ksub;
  const long long sK = (long long)ks * ks;
  const int* ke = c.sc->k_eff;
  eig_prod(c, false, false, ks, ks, ks, Tm, ks, sK, Wm, ks, sK, c.T2k, ks, sK, 3, ke, ke, ke);
  eig_prod(c, true, false, ks, ks, ks, Wm, ks, sK, c.T2k, ks, sK, Tm, ks, sK, 3, ke, ke, ke);
}

// Rayleigh-Ritz refinement: one FP32 Jacobi pass on the graded T (rotations accumulated in FP32,
// returned in FP64), one Newton-Schulz re-orthonormalisation of the accumulated rotation, one
// rotation of the basis and one FP64 congruence of T.  The basis Qa from the block Gram-Schmidt
// is orthonormal to working precision, so the loss of orthogonality of Qa W is that of W (FP32
// rotations): E = W^T W - I, M = I - E/2 + 3/8 E^2, and the final basis is Qa (W M) — k x k
// products, one n x k product.  The diagonal of the final T = (W M)^T T (W M), formed in FP64,
// gives the eigenvalues of the rank rule: the Jacobi pass stops when every off-diagonal entry is
// below JACOBI_TOL times the geometric mean of its two diagonal entries, so each diagonal entry
// differs from its eigenvalue by second order in that bound (relative 1e-8 and below), and a
// retained and a discarded direction mix by an angle that weighs the discarded energy, which is
// below the eps budget already.
static int refine(Ctx& c, double*& Qa, double*& Qb) {
  const int n = c.n, ks = c.ksub;
  const long long sQ = (long long)n * ks, sK = (long long)ks * ks;
  const int* ke = c.sc->k_eff;
  // one pass: T -> W^T T W (the FP32 rotations accumulated in W)
  if (ks <= JF_KMAX) {
    const size_t shm = 3ull * ks * (ks + 1) * sizeof(float);
    jacobi32f_kernel<<<3, JF_THREADS, shm, c.stream>>>(c.T, c.W, ks, c.sc, JACOBI_SWEEPS, JACOBI_TOL);
  } else {
    const size_t shm = 2ull * ks * (ks + 1) * sizeof(float);
    jacobi32_kernel<<<3, 1024, shm, c.stream>>>(c.T, c.W, ks, c.sc, JACOBI_SWEEPS, JACOBI_TOL);
  }
  // W2 = E = W^T W - I ; T2k = E^2 ; W2 = M
  eig_prod(c, true, false, ks, ks, ks, c.W, ks, sK, c.W, ks, sK, c.W2, ks, sK, 3, ke, ke, ke);
  dim3 g2((ks * ks + 255) / 256, 3);
  sub_identity_kernel<<<g2, 256, 0, c.stream>>>(c.W2, ks, c.sc);
  eig_prod(c, false, false, ks, ks, ks, c.W2, ks, sK, c.W2, ks, sK, c.T2k, ks, sK, 3, ke, ke, ke);
  ns_matrix_kernel<<<g2, 256, 0, c.stream>>>(c.W2, c.T2k, c.W2, ks, c.sc);
  // WM = W M (in the free product buffer Y) ; Qb = Qa (W M) ; T = (W M)^T T (W M)
  double* WM = c.Y;
  eig_prod(c, false, false, ks, ks, ks, c.W, ks, sK, c.W2, ks, sK, WM, ks, sK, 3, ke, ke, ke);
  eig_prod(c, false, false, n, ks, ks, Qa, ks, sQ, WM, ks, sK, Qb, ks, sQ, 3, nullptr, ke, ke);
  congruence(c, c.T, WM);
  std::swap(Qa, Qb);
  return 1 + 1 + 1 + 1 + 1 + 1 + 1 + 2;
}

int launch_subspace(Ctx& c) {
  const int n = c.n, ks = c.ksub;
  const long long sQ = (long long)n * ks, sK = (long long)ks * ks, sG = (long long)n * n;
  // X = G * Omega with the sparse sign embedding of this context
  // (the row shares of the traces go to the block Gram-Schmidt's partial-sum buffer, which is
  // free until that kernel starts)
  sparse_range_kernel<<<dim3(1, n, 3), KSUB_MAX, 0, c.stream>>>(c.G, c.om_colptr, c.om_row, c.om_sgn, n,
                                                               ks, c.X, c.part);
  traces_kernel<<<3, 256, 0, c.stream>>>(c.part, n, c.sc);
  // block Gram-Schmidt (cooperative)
  {
    void* args[] = {(void*)&c.X, (void*)&c.Q, (void*)&c.part, (void*)&n, (void*)&ks, (void*)&c.sc};
    const size_t shm = sizeof(double) * (size_t)((n + NBC - 1) / NBC) * ks;
    cudaLaunchCooperativeKernel((void*)bcgs2_kernel, dim3(3 * NBC), dim3(256), args, shm, c.stream);
  }
  const int* ke = c.sc->k_eff;
  // Y = G Q ; T = Q^T Y
  eig_prod(c, false, false, n, ks, n, c.G, n, sG, c.Q, ks, sQ, c.Y, ks, sQ, 3, nullptr, ke, nullptr);
  eig_prod(c, true, false, ks, ks, n, c.Q, ks, sQ, c.Y, ks, sQ, c.T, ks, sK, 3, ke, ke, nullptr);
  // Rayleigh-Ritz refinement; the rotated basis ends in c.X
  double* Qa = c.Q;
  double* Qb = c.X;
  int k = 5;                    // range finder, traces, Gram-Schmidt, two products
  k += refine(c, Qa, Qb);
  // Qa holds the final basis
  rank_select_kernel<<<3, 128, 0, c.stream>>>(c.T, ks, c.cfg.eps, c.cfg.rank_cap, c.rmax, c.order,
                                              c.ev, c.sc);
  long long totZ = 3ll * n * c.rmax;
  gather_Z_kernel<<<(unsigned)((totZ + 255) / 256), 256, 0, c.stream>>>(Qa, c.order, n, ks, c.rmax,
                                                                        c.sc, c.Z64, c.Z32);
  return k + 2;
}

cudaError_t set_attributes_eigen(int optin) {
  cudaError_t e = allow_max_dynamic_smem((const void*)jacobi32_kernel, optin);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)jacobi32f_kernel, optin);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)bcgs2_kernel, optin);
  return e;
}

}  // namespace rs
