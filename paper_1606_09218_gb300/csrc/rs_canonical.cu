// Tucker-to-canonical transform of the long-range part: the RS-canonical format (Def. 3.7) and
// its point values (Lemma 3.8).
//
//   beta[a, :, :] = sum_m s_{a,m} x_{a,m} y_{a,m}^T      one-sided Jacobi SVD of every mode-1 slice
//   the (a, m) terms except the smallest s^2 whose sum stays <= eps^2 ||beta||_F^2 are kept
//   u1 = V1[:, a], u2 = V2 x_{a,m}, u3 = V3 y_{a,m}, xi = s_{a,m}
//
// With orthonormal Tucker bases the Frobenius error of the long part is sqrt(discarded) <=
// eps ||beta||_F.  Sec. 3 reports RS-canonical ranks after a Tucker-to-canonical step of a given
// accuracy without stating its algorithm; the slice SVD is the reading taken.  A point value
// costs 3 R* products plus the windows of the neighbours, instead of r1 r2 for the Tucker form.
// FP64 throughout (the core and the bases are FP64 on every path).
#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr int CN_THREADS = 256;
constexpr int CN_MAX_SWEEPS = 40;
constexpr int CN_SORT_THREADS = 1024;

}  // namespace

// One CTA per slice a: one-sided Jacobi on the r2 x r3 matrix beta[a] (its r3 columns stored
// contiguously, A[c][b]; a zero column pads r3 to an even count), rotations accumulated in V
// (cp x cp, columns contiguous).  Round-robin pairs of columns, one warp per pair; a pair with
// |a_p . a_q| <= 1e-14 ||a_p|| ||a_q|| is not rotated, and a sweep without a rotation ends the
// iteration (at most CN_MAX_SWEEPS sweeps).  Writes s (sig[a][c]), x = A[:, c] / s and y = V[:, c].
__global__ void __launch_bounds__(CN_THREADS)
t2c_svd_kernel(const double* __restrict__ beta64, int rmax, const DevScalars* sc, double* sig, double* X,
               double* Y) {
  extern __shared__ double cn_smem[];
  __shared__ int s_rot;
  const int a = blockIdx.x;
  const int r1 = sc->rank[0], r2 = sc->rank[1], r3 = sc->rank[2];
  if (a >= r1) return;
  const int cp = r3 + (r3 & 1);
  double* A = cn_smem;                       // [cp][r2]
  double* V = A + (size_t)cp * r2;           // [cp][cp]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = CN_THREADS / 32;
  for (int e = tid; e < cp * r2; e += CN_THREADS) {
    const int cc = e / r2, b = e % r2;
    A[e] = cc < r3 ? beta64[((long long)a * rmax + b) * rmax + cc] : 0.0;
  }
  for (int e = tid; e < cp * cp; e += CN_THREADS) V[e] = (e / cp == e % cp) ? 1.0 : 0.0;
  __syncthreads();
  const int half = cp / 2;
  for (int sweep = 0; sweep < CN_MAX_SWEEPS && cp > 1; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < cp - 1; ++round) {
      for (int m = warp; m < half; m += nw) {
        const int p0 = (m == 0) ? 0 : 1 + (m - 1 + round) % (cp - 1);
        const int q0 = 1 + (cp - 2 - m + round) % (cp - 1);
        const int p = min(p0, q0), q = max(p0, q0);
        double* Ap = A + (size_t)p * r2;
        double* Aq = A + (size_t)q * r2;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int b = lane; b < r2; b += 32) {
          const double x = Ap[b], y = Aq[b];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {        // butterfly: every lane holds the sums
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (!(fabs(ga) > 1e-14 * sqrt(al * be))) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
        const double cs = 1.0 / sqrt(fma(t, t, 1.0)), sn = cs * t;
        for (int b = lane; b < r2; b += 32) {
          const double x = Ap[b], y = Aq[b];
          Ap[b] = cs * x - sn * y;
          Aq[b] = sn * x + cs * y;
        }
        double* Vp = V + (size_t)p * cp;
        double* Vq = V + (size_t)q * cp;
        for (int b = lane; b < cp; b += 32) {
          const double x = Vp[b], y = Vq[b];
          Vp[b] = cs * x - sn * y;
          Vq[b] = sn * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  for (int cc = warp; cc < r3; cc += nw) {
    const double* Ac = A + (size_t)cc * r2;
    double s2 = 0.0;
    for (int b = lane; b < r2; b += 32) s2 = fma(Ac[b], Ac[b], s2);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const double s = sqrt(s2);
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    const long long o = ((long long)a * rmax + cc) * rmax;
    for (int b = lane; b < r2; b += 32) X[o + b] = Ac[b] * inv;
    for (int d = lane; d < r3; d += 32) Y[o + d] = V[(size_t)cc * cp + d];
    if (lane == 0) sig[(long long)a * rmax + cc] = s;
  }
}

// Selection (one CTA): the r1 r3 squared singular values sorted ascending (bitonic, ties by
// index), the smallest discarded while their running sum stays <= eps^2 ||beta||_F^2 (the sum
// taken in that order, as the definition reads), the kept terms listed in (a, c) order.
// kept[k] = a * r3 + c, *count = R*.
__global__ void __launch_bounds__(CN_SORT_THREADS)
t2c_select_kernel(const double* __restrict__ sig, int rmax, const DevScalars* sc, double eps, int P, int* kept,
                  int* count) {
  extern __shared__ double sel_smem[];
  double* key = sel_smem;                        // [P]
  int* id = (int*)(key + P);                     // [P]
  __shared__ int s_ndisc;
  __shared__ int scan[CN_SORT_THREADS];
  const int r1 = sc->rank[0], r3 = sc->rank[2];
  const int M = r1 * r3, tid = threadIdx.x;
  for (int e = tid; e < P; e += CN_SORT_THREADS) {
    if (e < M) {
      const double s = sig[(long long)(e / r3) * rmax + e % r3];
      key[e] = s * s;
    } else {
      key[e] = __longlong_as_double(0x7ff0000000000000ll);   // +inf pads
    }
    id[e] = e;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int e = tid; e < P; e += CN_SORT_THREADS) {
        const int f = e ^ j;
        if (f > e) {
          const bool up = (e & k) == 0;
          const double ke = key[e], kf = key[f];
          const int ie = id[e], iff = id[f];
          const bool gt = (ke > kf) || (ke == kf && ie > iff);
          if (gt == up) {
            key[e] = kf; key[f] = ke;
            id[e] = iff; id[f] = ie;
          }
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    double tot = 0.0;
    for (int a = 0; a < r1; ++a) tot += sc->beta_a2[a];
    const double budget = eps * eps * tot;
    double cs = 0.0;
    int nd = 0;
    while (nd < M) {
      cs += key[nd];
      if (!(cs <= budget)) break;
      ++nd;
    }
    s_ndisc = nd;
  }
  __syncthreads();
  const int nd = s_ndisc;
  // key[] now flags the discarded terms by their original index
  for (int e = tid; e < P; e += CN_SORT_THREADS) key[e] = 0.0;
  __syncthreads();
  for (int e = tid; e < nd; e += CN_SORT_THREADS) key[id[e]] = 1.0;
  __syncthreads();
  const int per = (M + CN_SORT_THREADS - 1) / CN_SORT_THREADS;
  const int b0 = min(M, tid * per), b1 = min(M, b0 + per);
  int cnt = 0;
  for (int e = b0; e < b1; ++e) cnt += key[e] == 0.0 ? 1 : 0;
  scan[tid] = cnt;
  __syncthreads();
  for (int o = 1; o < CN_SORT_THREADS; o <<= 1) {
    const int v = tid >= o ? scan[tid - o] : 0;
    __syncthreads();
    scan[tid] += v;
    __syncthreads();
  }
  int pos = scan[tid] - cnt;
  for (int e = b0; e < b1; ++e)
    if (key[e] == 0.0) kept[pos++] = e;
  if (tid == CN_SORT_THREADS - 1) *count = scan[tid];
}

// Side matrices of the canonical form, U_l[i][k] (row length ld): u1 = V1[:, a], u2 = V2 x,
// u3 = V3 y; xi[k] = s.  Grid: (k blocks, i, l).
__global__ void __launch_bounds__(128)
t2c_factors_kernel(const double* __restrict__ Z64, int n, int rmax, const DevScalars* sc, const double* __restrict__ sig,
                   const double* __restrict__ X, const double* __restrict__ Y, const int* __restrict__ kept,
                   const int* __restrict__ count, int ld, double* U, double* xi) {
  const int k = blockIdx.x * 128 + threadIdx.x, i = blockIdx.y, l = blockIdx.z;
  if (k >= *count) return;
  const int r2 = sc->rank[1], r3 = sc->rank[2];
  const int e = kept[k], a = e / r3, cc = e % r3;
  const double* Vi = Z64 + ((long long)l * n + i) * rmax;
  const long long o = ((long long)a * rmax + cc) * rmax;
  double v;
  if (l == 0) {
    v = Vi[a];
    if (i == 0) xi[k] = sig[(long long)a * rmax + cc];
  } else if (l == 1) {
    v = 0.0;
    for (int b = 0; b < r2; ++b) v = fma(Vi[b], X[o + b], v);
  } else {
    v = 0.0;
    for (int d = 0; d < r3; ++d) v = fma(Vi[d], Y[o + d], v);
  }
  U[((long long)l * n + i) * ld + k] = v;
}

// Point values of the RS-canonical tensor (Lemma 3.8): sum_k xi_k U1[i1][k] U2[i2][k] U3[i3][k]
// plus the windows of the neighbours; one warp per point, indices clamped to the grid.
__global__ void __launch_bounds__(256)
canonical_eval_kernel(DevView c, const double* __restrict__ xi, const double* __restrict__ U, int ld,
                      const int* __restrict__ count, int M, const int* __restrict__ idx, double* out) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m = blockIdx.x * 8 + warp;
  if (m >= M) return;
  const int n = c.n;
  const int i1 = min(max(idx[3 * m], 0), n - 1), i2 = min(max(idx[3 * m + 1], 0), n - 1),
            i3 = min(max(idx[3 * m + 2], 0), n - 1);
  const double* u1 = U + (long long)i1 * ld;
  const double* u2 = U + ((long long)n + i2) * ld;
  const double* u3 = U + (2ll * n + i3) * ld;
  const int R = *count;
  double v = 0.0;
  for (int k = lane; k < R; k += 32) v = fma(xi[k] * u1[k], u2[k] * u3[k], v);
  window_add(c, i1, i2, i3, lane, v);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) out[m] = v;
}

size_t canonical_svd_smem(int r) {
  const size_t cp = (size_t)(r + (r & 1));
  return sizeof(double) * (cp * r + cp * cp);
}

size_t canonical_select_smem(int P) { return (sizeof(double) + sizeof(int)) * (size_t)P; }

int launch_canonical(Ctx& c, double eps, int r1, int r2, int r3, int P) {
  (void)r2;
  const int rm = r2 > r3 ? r2 : r3;
  t2c_svd_kernel<<<r1, CN_THREADS, canonical_svd_smem(rm), c.stream>>>(c.beta64, c.rmax, c.sc, c.cn_sig, c.cn_X,
                                                                       c.cn_Y);
  t2c_select_kernel<<<1, CN_SORT_THREADS, canonical_select_smem(P), c.stream>>>(c.cn_sig, c.rmax, c.sc, eps, P,
                                                                                c.cn_kept, c.cn_count);
  const dim3 grid((unsigned)((c.cn_cap + 127) / 128), (unsigned)c.n, 3);
  t2c_factors_kernel<<<grid, 128, 0, c.stream>>>(c.Z64, c.n, c.rmax, c.sc, c.cn_sig, c.cn_X, c.cn_Y, c.cn_kept,
                                                 c.cn_count, c.cn_cap, c.cn_U, c.cn_xi);
  return 3;
}

int launch_canonical_eval(Ctx& c, int M, const int* idx, double* out) {
  if (M <= 0) return 0;
  canonical_eval_kernel<<<(M + 7) / 8, 256, 0, c.stream>>>(make_view(c), c.cn_xi, c.cn_U, c.cn_cap, c.cn_count, M,
                                                          idx, out);
  return 1;
}

cudaError_t set_attributes_canonical(int optin) {
  cudaError_t e = allow_max_dynamic_smem((const void*)t2c_svd_kernel, optin);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)t2c_select_kernel, optin);
  return e;
}

}  // namespace rs
