// Setup stage: sinc quadrature and reference factors (Sec. 2.2), range split and window
// width (Sec. 2.3), particle snapping and aggregation, and the Gram matrices of the
// long-range side matrices (Sec. 3.2, Eq. (3.5); Sec. 6, step (I)).
#include "rs_internal.cuh"

namespace rs {

// ------------------------------------------------------------------ factors (a1, a2)
// p_k[d] = a_k^{1/3} * (1/h) int_{dh-h/2}^{dh+h/2} exp(-t_k^2 x^2) dx,  d = -(n-1)..(n-1)
// with t_k = exp(u0 + k h_q), a_k = (2/sqrt(pi)) h_q t_k (exponential sinc rule of the
// Laplace-Gauss transform of 1/z, Eqs. (2.6)-(2.8); Galerkin cell averages, Eq. (2.5)).
// dp_k[d] = d/dc of p_k at the centre offset c = d*h: a_k^{1/3} (exp(-t_k^2 (c+h/2)^2) -
// exp(-t_k^2 (c-h/2)^2)) / h (the cell average differentiated in its centre; adjoint forces).
// Any output pointer but pk64 may be null (that copy is then not written).
__global__ void factors_kernel(double* pk64, float* pk32, float* pk32lo, double* dpk64, float* dpk32, int R,
                               int n, double h, double hq, double u0) {
  const int L = 2 * n - 1;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= R * L) return;
  int k = e / L, di = e % L;
  double t = exp(u0 + k * hq);
  double a = 1.1283791670955126 * hq * t;          // 2/sqrt(pi)
  double cs = (double)(di - (n - 1)) * h;
  double c = fabs(cs);
  double lo = t * (c - 0.5 * h), hi = t * (c + 0.5 * h);
  double diff = (lo > 0.5) ? (erfc(lo) - erfc(hi)) : (erf(hi) - erf(lo));
  double ca = cbrt(a);
  double v = ca * (0.88622692545275801 / (t * h)) * diff;   // sqrt(pi)/2
  pk64[e] = v;
  if (pk32) pk32[e] = (float)v;
  if (pk32lo) pk32lo[e] = (float)(v - (double)(float)v);    // pk32 + pk32lo = p_k to 2^-48
  if (!dpk64 && !dpk32) return;                              // the caller needs no derivatives
  const double up = t * (cs + 0.5 * h), dn = t * (cs - 0.5 * h);
  const double dv = ca * (exp(-up * up) - exp(-dn * dn)) / h;
  if (dpk64) dpk64[e] = dv;
  if (dpk32) dpk32[e] = (float)dv;
}

// P_R(0), P_{R_l}(0), delta and the window half-width gamma (one CTA).
// gamma = #{g in [0, n-2] : sum_{k short} p_k[g+1] p_k[0]^2 > delta}  (the sum decreases in g)
__global__ void scalars_kernel(const double* pk64, int R, int R_l, int n, double delta_rel,
                               DevScalars* sc) {
  const int L = 2 * n - 1, c0 = n - 1;
  __shared__ double sPR0, sPRl0;
  __shared__ int cnt;
  if (threadIdx.x < 32) {
    // one warp loads the factors at the centre (32 at a time); lane 0 adds the cubes in the
    // order k = 0, 1, ... (the order of the host's window-width computation)
    const int lane = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int k0 = 0; k0 < R; k0 += 32) {
      const double v = (k0 + lane < R) ? pk64[(k0 + lane) * L + c0] : 0.0;
      for (int q = 0; q < 32 && k0 + q < R; ++q) {
        const double w = __shfl_sync(0xffffffffu, v, q);
        a += w * w * w;
        if (k0 + q < R_l) b += w * w * w;
      }
    }
    if (lane == 0) {
      sPR0 = a;
      sPRl0 = b;
      cnt = 0;
    }
  }
  __syncthreads();
  const double delta = delta_rel * sPR0;
  int local = 0;
  for (int g = threadIdx.x; g <= n - 2; g += blockDim.x) {
    double v = 0.0;
    for (int k = R_l; k < R; ++k) {
      double p0 = pk64[k * L + c0];
      v += pk64[k * L + c0 + g + 1] * p0 * p0;
    }
    if (v > delta) ++local;
  }
  atomicAdd(&cnt, local);
  __syncthreads();
  if (threadIdx.x == 0) {
    sc->P_R0 = sPR0;
    sc->P_Rl0 = sPRl0;
    sc->delta = delta;
    sc->gamma = min(cnt, n - 1);
  }
}

int launch_factors(Ctx& c) {
  int tot = c.R * c.L;
  // 64-thread CTAs: the FP64 special functions are bound by each SM's FP64 pipe, so the work is
  // spread over every SM instead of a hundred
  factors_kernel<<<(tot + 63) / 64, 64, 0, c.stream>>>(c.pk64, c.pk32, c.pk32lo, c.dpk64, c.dpk32, c.R, c.n,
                                                       c.h, c.cfg.h_q, c.cfg.u0);
  scalars_kernel<<<1, 256, 0, c.stream>>>(c.pk64, c.R, c.R_l, c.n, c.cfg.delta_rel, c.sc);
  return 2;
}

// ------------------------------------------------------------------ particles
// Snap each centre to its nearest grid point (ties away from zero; Sec. 3.2 places the
// centres on grid points), flag centres outside the box, and record the largest squared column
// weight w^2 = |z|^{2/3} (the scale of the aggregation below).
__device__ __forceinline__ bool snap_particle(const double* xyz, double z, int p, int n, double b, double h,
                                              int jj[3]) {
  bool bad = !isfinite(z);
  for (int l = 0; l < 3; ++l) {
    double x = xyz[3 * p + l];
    if (!isfinite(x) || fabs(x) > b * (1.0 + 1e-12)) bad = true;
    double s = (x + b) / h;
    int q = isfinite(s) ? (int)floor(s + 0.5) : 0;
    jj[l] = min(max(q, 0), n - 1);
  }
  return !bad;
}

__global__ void prepare_kernel(const double* xyz, const double* Z, int N, int n, double b,
                               double h, int* j, DevScalars* sc) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const double z = Z[p];
  int jj[3];
  const bool ok = snap_particle(xyz, z, p, n, b, h, jj);
  for (int l = 0; l < 3; ++l) j[3 * p + l] = jj[l];
  if (!ok) atomicOr(&sc->flags, (unsigned)FLAG_OUTSIDE);
  // the largest w^2 of the warp first (bits of non-negative doubles order as their values), one
  // atomic per warp instead of one per particle on a single address
  unsigned long long wb = (ok && z != 0.0) ? (unsigned long long)__double_as_longlong(pow(fabs(z), 2.0 / 3.0)) : 0ull;
  const unsigned act = __activemask();
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(act, wb, o);
    const int src = (threadIdx.x & 31) ^ o;
    if ((act >> src) & 1u) wb = u > wb ? u : wb;
  }
  if ((threadIdx.x & 31) == __ffs(act) - 1 && wb != 0ull) atomicMax(&sc->w2max_bits, wb);
}

// The weights C_l[j] = sum_{nu at j} w_nu^2 per grid coordinate (columns at equal shifts add in
// U U^T) as 64-bit fixed-point sums with the scale 2^e, N max w^2 2^e < 2^61: integer additions
// are exact, so C does not depend on the order of the atomics (a nonzero weight adds at least
// one unit, so no charged coordinate drops out).  C holds the integers until compact_nzj_kernel.
__device__ __forceinline__ int c_fx_shift(const DevScalars* sc, int N) {
  const double wmax = __longlong_as_double((long long)sc->w2max_bits);
  const double B = (double)N * wmax;
  if (!(B > 0.0) || !isfinite(B)) return 0;
  int E = 0;
  frexp(B, &E);
  return max(-1000, min(1000, 61 - E));
}

__global__ void aggregate_kernel(const double* xyz, const double* Z, int N, int n, double b, double h,
                                 double* C, const DevScalars* sc) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const double z = Z[p];
  int jj[3];
  if (!snap_particle(xyz, z, p, n, b, h, jj) || z == 0.0) return;
  const long long v = __double2ll_rn(pow(fabs(z), 2.0 / 3.0) * ldexp(1.0, c_fx_shift(sc, N)));
  unsigned long long* Cfx = reinterpret_cast<unsigned long long*>(C);
  for (int l = 0; l < 3; ++l) atomicAdd(&Cfx[l * n + jj[l]], (unsigned long long)(v > 0 ? v : 1));
}

// Deterministic compaction of the particles with nonzero charge (one CTA, chunked scan).
__global__ void compact_nz_kernel(const double* Z, int N, int* nz_idx, DevScalars* sc) {
  __shared__ int scan[1024];
  const int T = blockDim.x, t = threadIdx.x;
  const int per = (N + T - 1) / T;
  const int b0 = min(N, t * per), b1 = min(N, b0 + per);
  __shared__ double zred[32];
  int cnt = 0;
  double za = 0.0;
  for (int p = b0; p < b1; ++p) {
    const bool nz = Z[p] != 0.0 && isfinite(Z[p]);
    cnt += nz ? 1 : 0;
    za += nz ? fabs(Z[p]) : 0.0;
  }
  // sum |z| in a fixed order (bound of the core sums)
  for (int o = 16; o > 0; o >>= 1) za += __shfl_down_sync(0xffffffffu, za, o);
  if ((t & 31) == 0) zred[t >> 5] = za;
  scan[t] = cnt;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < (T + 31) / 32; ++w) s += zred[w];
    sc->zabs_sum = s;
  }
  for (int o = 1; o < T; o <<= 1) {
    int v = (t >= o) ? scan[t - o] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int pos = scan[t] - cnt;
  for (int p = b0; p < b1; ++p)
    if (Z[p] != 0.0 && isfinite(Z[p])) nz_idx[pos++] = p;
  if (t == T - 1) sc->n_nz = scan[t];
}

// Distinct coordinates with nonzero aggregated weight, per mode (one CTA per mode).
// The weights arrive as fixed-point integers (aggregate_kernel) and leave as FP64.
__global__ void compact_nzj_kernel(double* C, int n, int N, int* nzj, DevScalars* sc) {
  __shared__ int scan[1024];
  const int l = blockIdx.x, T = blockDim.x, t = threadIdx.x;
  double* Cl = C + l * n;
  const int per = (n + T - 1) / T;
  const int b0 = min(n, t * per), b1 = min(n, b0 + per);
  const double pinv = ldexp(1.0, -c_fx_shift(sc, N));
  int cnt = 0;
  for (int i = b0; i < b1; ++i) {
    const double v = (double)reinterpret_cast<const long long*>(Cl)[i] * pinv;
    Cl[i] = v;
    cnt += (v > 0.0) ? 1 : 0;
  }
  scan[t] = cnt;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    int v = (t >= o) ? scan[t - o] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int pos = scan[t] - cnt;
  for (int i = b0; i < b1; ++i)
    if (Cl[i] > 0.0) nzj[l * n + pos++] = i;
  if (t == T - 1) sc->nzj_count[l] = scan[t];
}

// Optional input check: any pair closer than min_sep (O(N^2), input coordinates).
__global__ void separation_kernel(const double* xyz, int N, double min_sep2, DevScalars* sc) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  double x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
  for (int q = p + 1; q < N; ++q) {
    double dx = xyz[3 * q] - x, dy = xyz[3 * q + 1] - y, dz = xyz[3 * q + 2] - z;
    if (dx * dx + dy * dy + dz * dz < min_sep2) {
      atomicOr(&sc->flags, (unsigned)FLAG_SEPARATION);
      return;
    }
  }
}

int launch_compact_nz(Ctx& c, int N) {
  compact_nz_kernel<<<1, 1024, 0, c.stream>>>(c.Z, N, c.nz_idx, c.sc);
  return 1;
}

int launch_prepare_particles(Ctx& c, int N, double min_sep, bool check_sep) {
  int k = 1;
  cudaMemsetAsync(c.C, 0, sizeof(double) * 3 * c.n, c.stream);
  if (N > 0) {
    prepare_kernel<<<(N + 255) / 256, 256, 0, c.stream>>>(c.xyz, c.Z, N, c.n, c.cfg.b, c.h, c.j, c.sc);
    aggregate_kernel<<<(N + 255) / 256, 256, 0, c.stream>>>(c.xyz, c.Z, N, c.n, c.cfg.b, c.h, c.C, c.sc);
    k += 2;
  }
  compact_nzj_kernel<<<3, 1024, 0, c.stream>>>(c.C, c.n, N, c.nzj, c.sc);
  if (check_sep && N > 1) {
    separation_kernel<<<(N + 127) / 128, 128, 0, c.stream>>>(c.xyz, N, min_sep * min_sep, c.sc);
    ++k;
  }
  return k;
}

// ------------------------------------------------------------------ F and Gram (a3, a4)
// F[a][b] = sum_{k long} p_k[a] p_k[b] over the doubled index range (L x L, FP64).
__global__ void fmatrix_kernel(const double* pk64, int R_l, int L, double* F) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  int a = blockIdx.y;
  if (b >= L) return;
  double v = 0.0;
  for (int k = 0; k < R_l; ++k) v += pk64[k * L + a] * pk64[k * L + b];
  F[(long long)a * L + b] = v;
}

// The same F for the double-float Gram, as FP32 pairs (hi, lo), from the factors as FP32 pairs:
// each product p_k[a] p_k[b] as hi*hi plus its exact rounding error plus the two cross terms,
// the R_l positive terms added by two-sums (relative error about 2^-46), no FP64 arithmetic.
// (a CTA takes FM_ROWS rows a and 256 columns b: each column's factors are loaded once for its
// rows, the rows' factors are staged in shared memory)
constexpr int FM_ROWS = 4;
__global__ void __launch_bounds__(256)
fmatrix_df_kernel(const float* __restrict__ ph, const float* __restrict__ pl, int R_l, int L, float2* F2) {
  __shared__ float2 pa[FM_ROWS][32];           // (hi, lo) of p_k[a] for the CTA's rows, 32 ranks k
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int a0 = blockIdx.y * FM_ROWS;
  float s[FM_ROWS], t[FM_ROWS];
#pragma unroll
  for (int r = 0; r < FM_ROWS; ++r) s[r] = t[r] = 0.f;
  for (int k0 = 0; k0 < R_l; k0 += 32) {
    const int nk = min(32, R_l - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < FM_ROWS * 32; e += blockDim.x) {
      const int r = e >> 5, k = e & 31, a = a0 + r;
      pa[r][k] = (a < L && k < nk) ? make_float2(ph[(k0 + k) * L + a], pl[(k0 + k) * L + a]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (b < L)
      for (int k = 0; k < nk; ++k) {
        const float xb = ph[(k0 + k) * L + b], yb = pl[(k0 + k) * L + b];
#pragma unroll
        for (int r = 0; r < FM_ROWS; ++r) {
          const float xa = pa[r][k].x, ya = pa[r][k].y;
          const float p = __fmul_rn(xa, xb);
          float e = fmaf(xa, xb, -p);
          e = fmaf(xa, yb, e);
          e = fmaf(ya, xb, e);
          const float u = __fadd_rn(s[r], p);
          const float z = __fsub_rn(u, s[r]);
          t[r] = __fadd_rn(t[r], __fadd_rn(__fadd_rn(__fsub_rn(s[r], __fsub_rn(u, z)), __fsub_rn(p, z)), e));
          s[r] = u;
        }
      }
  }
  if (b >= L) return;
#pragma unroll
  for (int r = 0; r < FM_ROWS; ++r) {
    const int a = a0 + r;
    if (a < L) {
      const float hi = __fadd_rn(s[r], t[r]);
      F2[(long long)a * L + b] = make_float2(hi, __fsub_rn(t[r], __fsub_rn(hi, s[r])));
    }
  }
}

static void launch_fmatrix(Ctx& c, bool split) {
  dim3 grid((c.L + 255) / 256, c.L);
  if (split)
    fmatrix_df_kernel<<<dim3((c.L + 255) / 256, (c.L + FM_ROWS - 1) / FM_ROWS), 256, 0, c.stream>>>(
        c.pk32, c.pk32lo, c.R_l, c.L, (float2*)c.F);
  else fmatrix_kernel<<<grid, 256, 0, c.stream>>>(c.pk64, c.R_l, c.L, c.F);
}

// G_l[i][i'] = sum_j C_l[j] F[i - j + n - 1][i' - j + n - 1]  (= U^(l) U^(l)^T with the columns
// of equal shift aggregated).  Upper-triangular 32x32 tiles; the transpose is mirrored.
__global__ void __launch_bounds__(256)
gram_kernel(const double* __restrict__ F, const double* __restrict__ C, const int* __restrict__ nzj,
            const DevScalars* sc, int n, double* G) {
  const int l = blockIdx.y;
  const int nt = (n + 31) / 32;
  // map blockIdx.x -> (ti <= tj); blockIdx.z takes half of the charged coordinates
  int t = blockIdx.x, ti = 0;
  while (t >= nt - ti) { t -= nt - ti; ++ti; }
  const int tj = ti + t;
  const int I0 = ti * 32, J0 = tj * 32;
  const int L = 2 * n - 1;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 8 rows of threads
  __shared__ double sw[256];
  __shared__ int sj[256];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int cnt_all = sc->nzj_count[l];
  const int split = gridDim.z;                 // 1: whole sum stored; 2: halves added
  const int mh = (cnt_all + split - 1) / split;
  const int mbeg = min(cnt_all, (int)blockIdx.z * mh), cnt = min(cnt_all, mbeg + mh);
  const double* Cl = C + l * n;
  const int* nl = nzj + l * n;
  const int ip = J0 + tx;
  for (int m0 = mbeg; m0 < cnt; m0 += 256) {
    int m = m0 + threadIdx.x;
    if (m < cnt) {
      int jv = nl[m];
      sj[threadIdx.x] = jv;
      sw[threadIdx.x] = Cl[jv];
    }
    __syncthreads();
    int mm = min(256, cnt - m0);
    for (int q = 0; q < mm; ++q) {
      int jv = sj[q];
      double w = sw[q];
      const double* Fr = F + (long long)(I0 + ty - jv + n - 1) * L + (ip - jv + n - 1);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int i = I0 + ty + 8 * r;
        if (i < n && ip < n) acc[r] = fma(w, Fr[(long long)(8 * r) * L], acc[r]);
      }
    }
    __syncthreads();
  }
  // with two halves, both add into the zeroed G: 0 + a + b in either order is the same sum
  double* Gl = G + (long long)l * n * n;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int i = I0 + ty + 8 * r;
    if (i < n && ip < n) {
      if (split == 1) {
        Gl[(long long)i * n + ip] = acc[r];
        if (ti != tj) Gl[(long long)ip * n + i] = acc[r];
      } else {
        atomicAdd(&Gl[(long long)i * n + ip], acc[r]);
        if (ti != tj) atomicAdd(&Gl[(long long)ip * n + i], acc[r]);
      }
    }
  }
}

// The FP32 bulk path forms G with the same sums in double-float arithmetic: w = C_l[j] and
// F as FP32 pairs (hi, lo), each product w F as hi*hi plus its exact rounding error (FMA) plus
// the two cross terms, added into an FP32 pair (s, t) by an error-free two-sum and renormalised
// every 16 terms.  All terms are positive, so every entry carries a relative error of order
// 2^-48 sqrt(terms) (about 1e-13; FP64 gives 1e-15), while the rank cut-off resolves eigenvalues
// down to eps^2/3 of the trace.  One FP64 FMA issues at 1/64 of the FP32 rate on this GPU, so the
// twelve FP32 operations of a term take a fifth of the time.  The exact roundings are
// intrinsics, so no product is contracted into an addition.
__global__ void __launch_bounds__(256)
gram_df_kernel(const float2* __restrict__ F2, const double* __restrict__ C, const int* __restrict__ nzj,
               const DevScalars* sc, int n, double* G) {
  const int l = blockIdx.y;
  const int nt = (n + 31) / 32;
  int t = blockIdx.x, ti = 0;
  while (t >= nt - ti) { t -= nt - ti; ++ti; }
  const int tj = ti + t;
  const int I0 = ti * 32, J0 = tj * 32;
  const int L = 2 * n - 1;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  __shared__ float2 sw[256];
  __shared__ int sj[256];
  float hs[4] = {0.f, 0.f, 0.f, 0.f}, ls[4] = {0.f, 0.f, 0.f, 0.f};
  const int cnt_all = sc->nzj_count[l];
  const int split = gridDim.z;
  const int mh = (cnt_all + split - 1) / split;
  const int mbeg = min(cnt_all, (int)blockIdx.z * mh), cnt = min(cnt_all, mbeg + mh);
  const double* Cl = C + l * n;
  const int* nl = nzj + l * n;
  const int ip = J0 + tx;
  bool live[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) live[r] = (I0 + ty + 8 * r < n) && ip < n;
  for (int m0 = mbeg; m0 < cnt; m0 += 256) {
    int m = m0 + threadIdx.x;
    if (m < cnt) {
      const int jv = nl[m];
      const double w = Cl[jv];
      const float wh = (float)w;
      sj[threadIdx.x] = jv;
      sw[threadIdx.x] = make_float2(wh, (float)(w - (double)wh));
    }
    __syncthreads();
    const int mm = min(256, cnt - m0);
    // one term w F into the pair (hs[r], ls[r])
    auto add_term = [&](int r, float2 w, float2 f) {
      const float p = __fmul_rn(w.x, f.x);
      float e = fmaf(w.x, f.x, -p);                   // exact error of the rounded product
      e = fmaf(w.x, f.y, e);
      e = fmaf(w.y, f.x, e);
      const float s = __fadd_rn(hs[r], p);            // two-sum: s + err = hs + p exactly
      const float z = __fsub_rn(s, hs[r]);
      const float err = __fadd_rn(__fsub_rn(hs[r], __fsub_rn(s, z)), __fsub_rn(p, z));
      ls[r] = __fadd_rn(ls[r], __fadd_rn(err, e));
      hs[r] = s;
    };
    auto renorm = [&]() {                             // fast two-sum, |hs| >= |ls|
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float s = __fadd_rn(hs[r], ls[r]);
        ls[r] = __fsub_rn(ls[r], __fsub_rn(s, hs[r]));
        hs[r] = s;
      }
    };
    auto row_ptr = [&](int jv) {
      return F2 + (long long)(I0 + ty - jv + n - 1) * L + (ip - jv + n - 1);
    };
    // four coordinates at a time: their 16 loads are issued before the sums (the order of the
    // additions, and the renormalisation every 16 terms, are those of one term at a time)
    int q = 0;
    for (; q + 4 <= mm; q += 4) {
      float2 f[4][4], w4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        w4[u] = sw[q + u];
        const float2* Fr = row_ptr(sj[q + u]);
#pragma unroll
        for (int r = 0; r < 4; ++r) f[u][r] = live[r] ? Fr[(long long)(8 * r) * L] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (live[r]) add_term(r, w4[u], f[u][r]);
        if (((q + u) & 15) == 15) renorm();
      }
    }
    for (; q < mm; ++q) {
      const float2 w = sw[q];
      const float2* Fr = row_ptr(sj[q]);
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (live[r]) add_term(r, w, Fr[(long long)(8 * r) * L]);
      if ((q & 15) == 15) renorm();
    }
    __syncthreads();
  }
  double* Gl = G + (long long)l * n * n;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int i = I0 + ty + 8 * r;
    if (!live[r]) continue;
    const double v = (double)hs[r] + (double)ls[r];
    if (split == 1) {
      Gl[(long long)i * n + ip] = v;
      if (ti != tj) Gl[(long long)ip * n + i] = v;
    } else {
      atomicAdd(&Gl[(long long)i * n + ip], v);
      if (ti != tj) atomicAdd(&Gl[(long long)ip * n + i], v);
    }
  }
}

int launch_gram_setup(Ctx& c) {
  launch_fmatrix(c, !c.fp64);                // double-float F on the FP32 bulk path
  cudaMemsetAsync(c.G, 0, sizeof(double) * 3 * (size_t)c.n * c.n, c.stream);
  return 1;
}

int launch_gram(Ctx& c) {
  const bool df = !c.fp64;                   // double-float sums on the FP32 bulk path
  int nt = (c.n + 31) / 32;
  dim3 grid(nt * (nt + 1) / 2, 3, 2);
  if (df) gram_df_kernel<<<grid, 256, 0, c.stream>>>((const float2*)c.F, c.C, c.nzj, c.sc, c.n, c.G);
  else gram_kernel<<<grid, 256, 0, c.stream>>>(c.F, c.C, c.nzj, c.sc, c.n, c.G);
  return 1;
}

}  // namespace rs
