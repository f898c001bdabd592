// Matrix-vector product with the RS interaction matrix of the grid (Sec. 4.1, problem (B),
// case (A)) and the interaction energy through it (Sec. 4.2, Eq. (4.6)).
//
// With the point set = the n^3 grid points, the interaction matrix of the reference kernel is
// a sum of Kronecker products of symmetric Toeplitz matrices,
//   A = sum_{k long} T_k (x) T_k (x) T_k  +  sum_{k short} T_k^g (x) T_k^g (x) T_k^g,
// T_k[i][i'] = p_k[i - i'] generated by the factor vector p_k, and T_k^g the same with the entries
// beyond the window |i - i'| > gamma set to zero (the short-range terms act only inside the
// window of Def. 3.4, so A applied to the charges is the long-range canonical sum plus the
// windows: the RS tensor before the Tucker truncation).  Each Kronecker term is applied as three
// mode products, and each mode product as 1-D circular convolutions of the fibres with the
// Toeplitz generator embedded in a circulant of size M (a power of two >= 2n - 2; the generator
// is even, so M = 2n - 2 needs no extra point), computed with FFTs: O(R n^3 log n) work for the
// n^3 x n^3 matrix.
//
// In FP32, for circulants of 32 to 2048 points, the mode products use a warp-level four-step
// FFT (mv_warp_kernel below).  Otherwise the FFTs are radix-2 in shared memory: 2B real fibres
// per CTA, packed two per complex
// sequence (the generator's transform is real, so the real and imaginary parts stay separate),
// bit-reversed on load, decimation in time forward, the symbol (transform of the generator,
// divided by M) applied in natural order, decimation in frequency with conjugate twiddles
// backward, read back in bit-reversed order.  The symbols are computed once per context in
// FP64 from the factor vectors (direct cosine sums with exact argument reduction).
#include "rs_internal.cuh"

#include <cmath>
#include <string>

namespace rs {

namespace {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// symbol[k][m] = (1/M) sum_{d=-(n-1)}^{n-1} c_k[d] cos(2 pi m d / M): the DFT of the circulant
// generator of T_k (real: the generator is even), c_k[d] = p_k[d], zero beyond gamma for the
// short terms; with M = 2n - 2 the offsets +-(n-1) are the same circulant entry, counted once.
__global__ void mv_symbol_kernel(const double* __restrict__ pk64, int R, int R_l, int n, int M,
                                 const DevScalars* sc, void* sym, bool fp64) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (m >= M) return;
  const int L = 2 * n - 1;
  const double* row = pk64 + (long long)k * L + n - 1;
  const int dmax = (k >= R_l) ? min(sc->gamma, n - 1) : n - 1;
  double s = row[0];
  for (int d = 1; d <= dmax; ++d) {
    const long long q = ((long long)m * d) % M;
    const double mult = (2 * d == M) ? 1.0 : 2.0;
    s += mult * row[d] * cospi(2.0 * (double)q / (double)M);
  }
  s /= (double)M;
  if (fp64) ((double*)sym)[(long long)k * M + m] = s;
  else ((float*)sym)[(long long)k * M + m] = (float)s;
}

// tw[q] = exp(-2 pi i q / M), q < M/2
__global__ void mv_twiddle_kernel(int M, void* tw, bool fp64) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= M / 2) return;
  double s, c;
  sincospi(2.0 * (double)q / (double)M, &s, &c);
  if (fp64) ((double2*)tw)[q] = make_double2(c, -s);
  else ((float2*)tw)[q] = make_float2((float)c, (float)-s);
}

// fibre f of axis `axis` of the C-order n^3 tensor: element i at base + i * stride
__device__ __forceinline__ void fibre(long long f, int axis, int n, long long& base, long long& stride) {
  const long long nn = (long long)n * n;
  if (axis == 2) { base = f * n; stride = 1; }
  else if (axis == 1) { base = (f / n) * nn + f % n; stride = n; }
  else { base = f; stride = nn; }
}

// Y (=, or += with accumulate) the Toeplitz product T_k along `axis` of X, by FFT convolution.
template <typename T>
__global__ void __launch_bounds__(256)
mv_mode_kernel(const T* __restrict__ X, T* __restrict__ Y, int n, int M, int logM, int B, int axis,
               const T* __restrict__ sym, const typename Cplx<T>::type* __restrict__ tw, int accumulate) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char mv_smem[];
  C* buf = reinterpret_cast<C*>(mv_smem);        // B sequences of M
  C* stw = buf + (size_t)B * M;                   // M/2 twiddles
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long nf = (long long)n * n;
  const long long f0 = (long long)blockIdx.x * 2 * B;
  const int nfl = 2 * B;
  const int half_M = M >> 1;
  for (int q = tid; q < half_M; q += nt) stw[q] = tw[q];
  for (int e = tid; e < B * M; e += nt) {
    C z;
    z.x = T(0);
    z.y = T(0);
    buf[e] = z;
  }
  __syncthreads();
  // load: fibre 2p -> real part, 2p + 1 -> imaginary part of sequence p, at bit-reversed index
  for (int e = tid; e < nfl * n; e += nt) {
    int fl, i;
    if (axis == 2) { fl = e / n; i = e % n; }
    else { fl = e % nfl; i = e / nfl; }            // consecutive fibres are adjacent in memory
    const long long f = f0 + fl;
    if (f >= nf) continue;
    long long base, stride;
    fibre(f, axis, n, base, stride);
    const T v = X[base + (long long)i * stride];
    const int pos = (int)(__brev((unsigned)i) >> (32 - logM));
    C* slot = buf + (size_t)(fl >> 1) * M + pos;
    if (fl & 1) slot->y = v;
    else slot->x = v;
  }
  __syncthreads();
  // forward transform, decimation in time (natural order out)
  for (int s = 1; s <= logM; ++s) {
    const int half = 1 << (s - 1);
    for (int e = tid; e < B * half_M; e += nt) {
      const int p = e / half_M, jb = e % half_M;
      const int pos = jb & (half - 1);
      const int i0 = ((jb >> (s - 1)) << s) + pos, i1 = i0 + half;
      C* b0 = buf + (size_t)p * M;
      const C w = stw[pos << (logM - s)];
      const C a = b0[i0];
      const C t = cmul(b0[i1], w);
      C u, v;
      u.x = a.x + t.x; u.y = a.y + t.y;
      v.x = a.x - t.x; v.y = a.y - t.y;
      b0[i0] = u;
      b0[i1] = v;
    }
    __syncthreads();
  }
  for (int e = tid; e < B * M; e += nt) {
    const T sv = sym[e % M];
    buf[e].x *= sv;
    buf[e].y *= sv;
  }
  __syncthreads();
  // inverse transform, decimation in frequency with conjugate twiddles (bit-reversed order out)
  for (int s = logM; s >= 1; --s) {
    const int half = 1 << (s - 1);
    for (int e = tid; e < B * half_M; e += nt) {
      const int p = e / half_M, jb = e % half_M;
      const int pos = jb & (half - 1);
      const int i0 = ((jb >> (s - 1)) << s) + pos, i1 = i0 + half;
      C* b0 = buf + (size_t)p * M;
      C w = stw[pos << (logM - s)];
      w.y = -w.y;
      const C a = b0[i0], b = b0[i1];
      C u, d;
      u.x = a.x + b.x; u.y = a.y + b.y;
      d.x = a.x - b.x; d.y = a.y - b.y;
      b0[i0] = u;
      b0[i1] = cmul(d, w);
    }
    __syncthreads();
  }
  for (int e = tid; e < nfl * n; e += nt) {
    int fl, i;
    if (axis == 2) { fl = e / n; i = e % n; }
    else { fl = e % nfl; i = e / nfl; }
    const long long f = f0 + fl;
    if (f >= nf) continue;
    long long base, stride;
    fibre(f, axis, n, base, stride);
    const int pos = (int)(__brev((unsigned)i) >> (32 - logM));
    const C* slot = buf + (size_t)(fl >> 1) * M + pos;
    const T v = (fl & 1) ? slot->y : slot->x;
    T* out = Y + base + (long long)i * stride;
    if (accumulate) *out += v;
    else *out = v;
  }
}

// The same mode product with a warp-level four-step FFT (M = 32 P): lane l holds v[q] = x[l + 32 q];
// a P-point DFT in registers over q, the twiddles W_M^(l k2), and a 32-point DFT across the lanes
// by shuffles (decimation in frequency: lane l ends with the frequency k2 + P brev5(l)); after the
// symbol, the inverse steps in reverse order (decimation in time across the lanes, conjugate
// twiddles, inverse register DFT).  No CTA barrier inside the transform.  A CTA handles 16
// fibres (two per warp); fibres along a strided axis are staged through shared memory so that
// global loads and stores stay coalesced.
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

template <typename C, int M>
__device__ __forceinline__ C twid(const C* stw, int q) {       // exp(-2 pi i q / M)
  q &= M - 1;
  C w = stw[q & (M / 2 - 1)];
  if (q >= M / 2) { w.x = -w.x; w.y = -w.y; }
  return w;
}

// in-register P-point DFT over the register index, natural order in and out
template <typename C, int P, bool INV>
__device__ __forceinline__ void reg_dft(C* v, const C* stw) {
  constexpr int M = 32 * P;
#pragma unroll
  for (int i = 0; i < P; ++i) {
    int j = 0;
#pragma unroll
    for (int b = 1, r = P >> 1; b < P; b <<= 1, r >>= 1)
      if (i & b) j |= r;
    if (i < j) { const C t = v[i]; v[i] = v[j]; v[j] = t; }
  }
#pragma unroll
  for (int half = 1; half < P; half <<= 1) {
#pragma unroll
    for (int g0 = 0; g0 < P; g0 += 2 * half) {
#pragma unroll
      for (int pos = 0; pos < half; ++pos) {
        C w = twid<C, M>(stw, pos * (M / (2 * half)));
        if (INV) w = cconj(w);
        const C a = v[g0 + pos], b = cmul(v[g0 + pos + half], w);
        v[g0 + pos] = cadd(a, b);
        v[g0 + pos + half] = csub(a, b);
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ T shfl_x(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

template <typename T, int P>
__global__ void __launch_bounds__(256)
mv_warp_kernel(const T* __restrict__ X, T* __restrict__ Y, int n, int axis, const T* __restrict__ sym,
               const typename Cplx<T>::type* __restrict__ tw, int accumulate) {
  using C = typename Cplx<T>::type;
  constexpr int M = 32 * P, FB = 16, LD = FB + 1;
  extern __shared__ __align__(16) unsigned char mv_smem[];
  C* stw = reinterpret_cast<C*>(mv_smem);
  T* tile = reinterpret_cast<T*>(stw + M / 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long nf = (long long)n * n;
  const long long f0 = (long long)blockIdx.x * FB;
  const bool strided = axis != 2;
  for (int q = tid; q < M / 2; q += 256) stw[q] = tw[q];
  if (strided) {
    for (int e = tid; e < n * FB; e += 256) {
      const int fl = e & (FB - 1), i = e >> 4;
      const long long f = f0 + fl;
      T v = T(0);
      if (f < nf) {
        long long base, stride;
        fibre(f, axis, n, base, stride);
        v = X[base + (long long)i * stride];
      }
      tile[i * LD + fl] = v;
    }
  }
  __syncthreads();
  const int fa = 2 * warp;
  const long long ga = f0 + fa;
  C v[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int i = lane + 32 * q;
    T re = T(0), im = T(0);
    if (i < n) {
      if (strided) {
        re = tile[i * LD + fa];
        im = tile[i * LD + fa + 1];
      } else {
        if (ga < nf) re = X[ga * n + i];
        if (ga + 1 < nf) im = X[(ga + 1) * n + i];
      }
    }
    v[q].x = re;
    v[q].y = im;
  }
  // forward: register DFT, twiddles, cross-lane DIF
  reg_dft<C, P, false>(v, stw);
#pragma unroll
  for (int q = 1; q < P; ++q) v[q] = cmul(v[q], twid<C, M>(stw, lane * q));
#pragma unroll
  for (int span = 16; span >= 1; span >>= 1) {
    const C w = twid<C, M>(stw, (lane & (span - 1)) * (16 / span) * P);
    const bool hi = (lane & span) != 0;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      C p;
      p.x = shfl_x(v[q].x, span);
      p.y = shfl_x(v[q].y, span);
      v[q] = hi ? cmul(csub(p, v[q]), w) : cadd(v[q], p);
    }
  }
  {
    int lb = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b)
      if (lane & (1 << b)) lb |= 16 >> b;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const T sv = sym[q + P * lb];
      v[q].x *= sv;
      v[q].y *= sv;
    }
  }
  // inverse: cross-lane DIT with conjugate twiddles, twiddles, register DFT
#pragma unroll
  for (int span = 1; span <= 16; span <<= 1) {
    const C w = cconj(twid<C, M>(stw, (lane & (span - 1)) * (16 / span) * P));
    const bool hi = (lane & span) != 0;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      C p;
      p.x = shfl_x(v[q].x, span);
      p.y = shfl_x(v[q].y, span);
      v[q] = hi ? csub(p, cmul(v[q], w)) : cadd(v[q], cmul(p, w));
    }
  }
#pragma unroll
  for (int q = 1; q < P; ++q) v[q] = cmul(v[q], cconj(twid<C, M>(stw, lane * q)));
  reg_dft<C, P, true>(v, stw);
  if (strided) {
    __syncthreads();                           // every warp has read its fibres from the tile
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = lane + 32 * q;
      if (i < n) {
        tile[i * LD + fa] = v[q].x;
        tile[i * LD + fa + 1] = v[q].y;
      }
    }
    __syncthreads();
    for (int e = tid; e < n * FB; e += 256) {
      const int fl = e & (FB - 1), i = e >> 4;
      const long long f = f0 + fl;
      if (f >= nf) continue;
      long long base, stride;
      fibre(f, axis, n, base, stride);
      T* out = Y + base + (long long)i * stride;
      const T val = tile[i * LD + fl];
      if (accumulate) *out += val;
      else *out = val;
    }
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int i = lane + 32 * q;
      if (i >= n) continue;
      if (ga < nf) {
        T* out = Y + ga * n + i;
        if (accumulate) *out += v[q].x;
        else *out = v[q].x;
      }
      if (ga + 1 < nf) {
        T* out = Y + (ga + 1) * n + i;
        if (accumulate) *out += v[q].y;
        else *out = v[q].y;
      }
    }
  }
}

template <typename T, int P>
void launch_mv_warp(const T* X, T* Y, int n, int axis, const T* sym, const typename Cplx<T>::type* tw,
                    int accumulate, cudaStream_t s) {
  const long long nf = (long long)n * n;
  const size_t smem = sizeof(typename Cplx<T>::type) * (16 * P) + sizeof(T) * (size_t)n * 17;
  mv_warp_kernel<T, P><<<(unsigned)((nf + 15) / 16), 256, smem, s>>>(X, Y, n, axis, sym, tw, accumulate);
}

// one mode product by the warp kernel when M = 32 P is one of its sizes; false otherwise
template <typename T>
bool mode_product_warp(int M, const T* X, T* Y, int n, int axis, const T* sym, const typename Cplx<T>::type* tw,
                       int accumulate, cudaStream_t s) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
  switch (M) {
    case 32: launch_mv_warp<T, 1>(X, Y, n, axis, sym, tw, accumulate, s); return true;
    case 64: launch_mv_warp<T, 2>(X, Y, n, axis, sym, tw, accumulate, s); return true;
    case 128: launch_mv_warp<T, 4>(X, Y, n, axis, sym, tw, accumulate, s); return true;
    case 256: launch_mv_warp<T, 8>(X, Y, n, axis, sym, tw, accumulate, s); return true;
    case 512: launch_mv_warp<T, 16>(X, Y, n, axis, sym, tw, accumulate, s); return true;
    case 1024: launch_mv_warp<T, 32>(X, Y, n, axis, sym, tw, accumulate, s); return true;
    case 2048:
      launch_mv_warp<T, 64>(X, Y, n, axis, sym, tw, accumulate, s);
      return true;
    default: return false;
  }
  }
}

// Y -= d X with d the diagonal of the selected terms (sum of p_k[0]^3 over them)
template <typename T>
__global__ void mv_offdiag_kernel(const T* X, T* Y, long long total, const DevScalars* sc, int which) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const double d = (which == 3) ? sc->P_R0 : (which == 1 ? sc->P_Rl0 : sc->P_R0 - sc->P_Rl0);
  Y[e] = (T)((double)Y[e] - d * (double)X[e]);
}

// charges onto the grid (the grid was zeroed): z at the particle's grid point
template <typename T>
__global__ void mv_scatter_kernel(const int* __restrict__ j, const double* __restrict__ Z, const int* nz_idx,
                                  const DevScalars* sc, int n, T* X) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= sc->n_nz) return;
  const int p = nz_idx[m];
  const long long o = ((long long)j[3 * p] * n + j[3 * p + 1]) * n + j[3 * p + 2];
  atomicAdd(X + o, (T)Z[p]);
}

// E = 1/2 sum_j z_j Y(x_j) (one CTA, fixed order)
template <typename T>
__global__ void mv_energy_kernel(const int* __restrict__ j, const double* __restrict__ Z, const int* nz_idx,
                                 const DevScalars* sc, int n, const T* Y, double* E) {
  __shared__ double red[32];
  const int nnz = sc->n_nz;
  const int per = (nnz + blockDim.x - 1) / blockDim.x;
  const int m0 = min(nnz, (int)threadIdx.x * per), m1 = min(nnz, m0 + per);
  double s = 0.0;
  for (int m = m0; m < m1; ++m) {
    const int p = nz_idx[m];
    const long long o = ((long long)j[3 * p] * n + j[3 * p + 1]) * n + j[3 * p + 2];
    s += Z[p] * (double)Y[o];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    *E = 0.5 * t;
  }
}

size_t mv_smem_bytes(const Ctx& c) {
  const size_t cs = c.fp64 ? sizeof(double2) : sizeof(float2);
  return cs * ((size_t)c.mv_B * c.mv_M + (size_t)c.mv_M / 2);
}

bool mv_alloc(Ctx& c, bool with_energy) {
  const size_t ts = c.fp64 ? 8 : 4;
  const size_t n3 = (size_t)c.n * c.n * c.n;
  if (!c.mv_sym) {
    int M = 1, logM = 0;
    while (M < 2 * c.n - 2) { M <<= 1; ++logM; }
    if (M < 2) { M = 2; logM = 1; }
    const size_t cs = c.fp64 ? sizeof(double2) : sizeof(float2);
    int B = (int)((64 * 1024) / (cs * M));
    if (B < 1) B = 1;
    if (B > 16) B = 16;
    c.mv_M = M;
    c.mv_logM = logM;
    c.mv_B = B;
    if (cudaMalloc(&c.mv_sym, ts * (size_t)c.R * M) != cudaSuccess ||
        cudaMalloc(&c.mv_tw, 2 * ts * (size_t)(M / 2 > 0 ? M / 2 : 1)) != cudaSuccess ||
        cudaMalloc(&c.mv_U, ts * n3) != cudaSuccess || cudaMalloc(&c.mv_V, ts * n3) != cudaSuccess) {
      cudaGetLastError();
      free_matvec(c);
      return false;
    }
    c.mv_symbols_ready = false;
  }
  if (with_energy && !c.mv_X) {
    if (cudaMalloc(&c.mv_X, ts * n3) != cudaSuccess || cudaMalloc(&c.mv_Y, ts * n3) != cudaSuccess ||
        cudaMalloc(&c.mv_E, sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      if (c.mv_X) cudaFree(c.mv_X);
      if (c.mv_Y) cudaFree(c.mv_Y);
      if (c.mv_E) cudaFree(c.mv_E);
      c.mv_X = c.mv_Y = nullptr;
      c.mv_E = nullptr;
      return false;
    }
  }
  return true;
}

template <typename T>
int matvec_t(Ctx& c, const T* X, T* Y, int which) {
  const int n = c.n, M = c.mv_M;
  int k = 0;
  if (!c.mv_symbols_ready) {
    mv_symbol_kernel<<<dim3((M + 255) / 256, c.R), 256, 0, c.stream>>>(c.pk64, c.R, c.R_l, n, M, c.sc, c.mv_sym,
                                                                        c.fp64);
    mv_twiddle_kernel<<<(M / 2 + 255) / 256, 256, 0, c.stream>>>(M, c.mv_tw, c.fp64);
    c.mv_symbols_ready = true;
    k += 2;
  }
  const long long nf = (long long)n * n;
  const unsigned grid = (unsigned)((nf + 2 * c.mv_B - 1) / (2 * c.mv_B));
  const size_t smem = mv_smem_bytes(c);
  using C = typename Cplx<T>::type;
  const T* sym = (const T*)c.mv_sym;
  const C* tw = (const C*)c.mv_tw;
  T* U = (T*)c.mv_U;
  T* V = (T*)c.mv_V;
  const int k0 = (which & 1) ? 0 : c.R_l, k1 = (which & 2) ? c.R : c.R_l;
  bool first = true;
  // FP32: the warp four-step FFT (measured 2x faster than the shared-memory radix-2 kernel on
  // a 513^3 grid); FP64: the shared-memory kernel (the warp kernel's FP64 shuffles made it
  // slower on a 129^3 grid)
  auto mode = [&](const T* in, T* out, int axis, const T* s, int acc) {
    if (sizeof(T) == 8 || !mode_product_warp<T>(M, in, out, n, axis, s, tw, acc, c.stream))
      mv_mode_kernel<T><<<grid, 256, smem, c.stream>>>(in, out, n, M, c.mv_logM, c.mv_B, axis, s, tw, acc);
  };
  for (int t = k0; t < k1; ++t) {
    const T* s = sym + (size_t)t * M;
    mode(X, U, 2, s, 0);
    mode(U, V, 1, s, 0);
    mode(V, Y, 0, s, first ? 0 : 1);
    first = false;
    k += 3;
  }
  if (first) {                                  // no term selected
    cudaMemsetAsync(Y, 0, sizeof(T) * (size_t)n * n * n, c.stream);
  }
  return k;
}

}  // namespace

void free_matvec(Ctx& c) {
  for (void* p : {c.mv_sym, c.mv_tw, c.mv_U, c.mv_V, c.mv_X, c.mv_Y, (void*)c.mv_E})
    if (p) cudaFree(p);
  c.mv_sym = c.mv_tw = c.mv_U = c.mv_V = c.mv_X = c.mv_Y = nullptr;
  c.mv_E = nullptr;
  c.mv_symbols_ready = false;
}

cudaError_t set_attributes_matvec(int optin) {
  const void* fs[] = {(const void*)mv_mode_kernel<float>, (const void*)mv_mode_kernel<double>,
                      (const void*)mv_warp_kernel<float, 1>, (const void*)mv_warp_kernel<float, 2>,
                      (const void*)mv_warp_kernel<float, 4>, (const void*)mv_warp_kernel<float, 8>,
                      (const void*)mv_warp_kernel<float, 16>, (const void*)mv_warp_kernel<float, 32>,
                      (const void*)mv_warp_kernel<float, 64>};
  cudaError_t e = cudaSuccess;
  for (const void* f : fs)
    if (e == cudaSuccess) e = allow_max_dynamic_smem(f, optin);
  return e;
}

// Y = A X (which: 1 long terms, 2 short terms, 3 both; offdiag: minus diag(A) X)
int launch_matvec(Ctx& c, const void* X, void* Y, int which, bool offdiag, std::string& err) {
  if (!mv_alloc(c, false)) {
    err = "matvec: device allocation failed";
    return -1;
  }
  int k = launch_factors(c);                    // factors and window width (depend on cfg only)
  k += c.fp64 ? matvec_t<double>(c, (const double*)X, (double*)Y, which)
              : matvec_t<float>(c, (const float*)X, (float*)Y, which);
  if (offdiag) {
    const long long tot = (long long)c.n * c.n * c.n;
    const unsigned g = (unsigned)((tot + 255) / 256);
    if (c.fp64) mv_offdiag_kernel<double><<<g, 256, 0, c.stream>>>((const double*)X, (double*)Y, tot, c.sc, which);
    else mv_offdiag_kernel<float><<<g, 256, 0, c.stream>>>((const float*)X, (float*)Y, tot, c.sc, which);
    ++k;
  }
  return k;
}

// E = 1/2 <(A - diag A) z, z> for the charges of the last solve (on their grid points)
int launch_energy_matvec(Ctx& c, std::string& err) {
  if (!mv_alloc(c, true)) {
    err = "energy_matvec: device allocation failed";
    return -1;
  }
  const int n = c.n;
  const size_t n3 = (size_t)n * n * n;
  int k = 0;
  cudaMemsetAsync(c.mv_X, 0, (c.fp64 ? 8 : 4) * n3, c.stream);
  const unsigned gb = (unsigned)((c.maxN + 255) / 256 > 0 ? (c.maxN + 255) / 256 : 1);
  if (c.fp64) mv_scatter_kernel<double><<<gb, 256, 0, c.stream>>>(c.j, c.Z, c.nz_idx, c.sc, n, (double*)c.mv_X);
  else mv_scatter_kernel<float><<<gb, 256, 0, c.stream>>>(c.j, c.Z, c.nz_idx, c.sc, n, (float*)c.mv_X);
  ++k;
  const int km = launch_matvec(c, c.mv_X, c.mv_Y, 3, true, err);
  if (km < 0) return -1;
  k += km;
  if (c.fp64) mv_energy_kernel<double><<<1, 1024, 0, c.stream>>>(c.j, c.Z, c.nz_idx, c.sc, n, (const double*)c.mv_Y, c.mv_E);
  else mv_energy_kernel<float><<<1, 1024, 0, c.stream>>>(c.j, c.Z, c.nz_idx, c.sc, n, (const float*)c.mv_Y, c.mv_E);
  return k + 1;
}

}  // namespace rs
