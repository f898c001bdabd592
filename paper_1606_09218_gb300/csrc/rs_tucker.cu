// Tucker stage: projection and core of the RHOSVD (Sec. 6, step (II), Eqs. (6.2)-(6.3)),
// full-grid reconstruction of the RS-Tucker tensor (Def. 3.9, Eq. (3.11)) with the
// short-range windows of the cumulated canonical tensor (Defs. 3.4, 3.6), and the point
// evaluation of Lemma 3.10 used for the interaction energy (Sec. 4.2, Eq. (4.7)).
#include "rs_internal.cuh"

#include <cstdlib>
#include <cstring>

namespace rs {

template <typename T> struct Bulk;
template <> struct Bulk<float> { static const float* pk(const Ctx& c) { return c.pk32; } static const float* Z(const Ctx& c) { return c.Z32; } };
template <> struct Bulk<double> { static const double* pk(const Ctx& c) { return c.pk64; } static const double* Z(const Ctx& c) { return c.Z64; } };

// ------------------------------------------------------------------ projection
// Qp[l][j][k][a] = sum_i Z_l[i][a] p_k[i - j]   (Z0^(l)^T applied to the shifted reference
// factors; the projected side matrix is U~^(l)[a, (nu,k)] = w_nu Qp[l][j_l^(nu)][k][a]).
template <typename T>
__global__ void __launch_bounds__(256)
proj_kernel(const T* __restrict__ Zb, const T* __restrict__ pk, int n, int rmax, int R_l,
            const DevScalars* sc, T* Qp) {
  const int l = blockIdx.z, k = blockIdx.y, j0 = blockIdx.x * 32;
  const int r = sc->rank[l];
  if (r == 0) return;
  const int L = 2 * n - 1;
  const int al = threadIdx.x % 32, jl = threadIdx.x / 32;
  const int na = (r + 31) / 32;     // a-groups in use (<= rmax/32)
  __shared__ T sZ[32][161];
  __shared__ T sp[64];
  T acc[4][5];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[s][q] = T(0);
  const T* Zl = Zb + (long long)l * n * rmax;
  const T* pkk = pk + (long long)k * L;
  for (int i0 = 0; i0 < n; i0 += 32) {
    for (int e = threadIdx.x; e < 32 * na * 32; e += 256) {
      int ii = e / (na * 32), a = e % (na * 32);
      int i = i0 + ii;
      sZ[ii][a] = (i < n && a < rmax) ? Zl[(long long)i * rmax + a] : T(0);
    }
    // p_k[i - j] for i in [i0, i0+32), j in [j0, j0+32): offsets i - j in [i0-j0-31, i0-j0+31]
    if (threadIdx.x < 63) {
      int d = i0 - j0 - 31 + threadIdx.x;
      int idx = d + n - 1;
      sp[threadIdx.x] = (idx >= 0 && idx < L) ? pkk[idx] : T(0);
    }
    __syncthreads();
    const int ilim = min(32, n - i0);
    for (int ii = 0; ii < ilim; ++ii) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        int jj = jl + 8 * s;                      // j = j0 + jj
        T f = sp[ii - jj + 31];
#pragma unroll
        for (int q = 0; q < 5; ++q)
          if (q < na) acc[s][q] = fma(sZ[ii][al + 32 * q], f, acc[s][q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int j = j0 + jl + 8 * s;
    if (j >= n) continue;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      int a = al + 32 * q;
      if (a < rmax && q < (rmax + 31) / 32)
        Qp[(((long long)l * n + j) * R_l + k) * rmax + a] = (a < r) ? acc[s][q] : T(0);
    }
  }
}

// ------------------------------------------------------------------ core
// beta[a][b][c] = sum_{p nonzero} z_p sum_{k long} Qp1[j1][k][a] Qp2[j2][k][b] Qp3[j3][k][c]
// (Eq. (6.2): beta = xi x_1 U~1 x_2 U~2 x_3 U~3 with xi = sign z and w^3 = |z|).
// CTA tile: 32 a x (8 b x 8 c); K = (particle, k) split over gridDim.y; FP32 products are
// summed in chunks of 64 K-elements and the chunks accumulated in FP64.
template <typename T>
__global__ void __launch_bounds__(256)
core_kernel(const T* __restrict__ Qp, const int* __restrict__ jidx, const int* __restrict__ nz_idx,
            const double* __restrict__ Z, int n, int rmax, int R_l, const DevScalars* sc,
            double* beta64) {
  const int r1 = sc->rank[0], r2 = sc->rank[1], r3 = sc->rank[2];
  const int ta = (rmax + 31) / 32, tb = (rmax + 7) / 8;
  int bt = blockIdx.x;
  const int tcI = bt % tb; bt /= tb;
  const int tbI = bt % tb; bt /= tb;
  const int taI = bt;
  if (taI >= ta) return;
  const int a0 = taI * 32, b0 = tbI * 8, c0 = tcI * 8;
  if (a0 >= r1 || b0 >= r2 || c0 >= r3) return;
  const int nnz = sc->n_nz;
  const long long Ktot = (long long)nnz * R_l;
  const long long per = (Ktot + gridDim.y - 1) / gridDim.y;
  const long long kb = blockIdx.y * per, ke = min(Ktot, kb + per);
  if (kb >= ke) return;
  __shared__ T sA[32][33];
  __shared__ T sB[32][8];
  __shared__ T sC[32][8];
  const int a = threadIdx.x % 32, bl = threadIdx.x / 32;     // b = b0 + bl; c loops
  T acc[8];
  double acc64[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) { acc[q] = T(0); acc64[q] = 0.0; }
  const long long sL = (long long)n * R_l * rmax;
  int chunk_count = 0;
  for (long long K0 = kb; K0 < ke; K0 += 32) {
    // stage 32 K-elements
    {
      int kk = threadIdx.x / 8, part = threadIdx.x % 8;   // 32 x 8 loaders
      long long K = K0 + kk;
      bool ok = K < ke;
      int p = ok ? nz_idx[K / R_l] : 0;
      int k = ok ? (int)(K % R_l) : 0;
      T z = ok ? (T)Z[p] : T(0);
      int j1 = jidx[3 * p], j2 = jidx[3 * p + 1], j3 = jidx[3 * p + 2];
      const T* q1 = Qp + (((long long)0 * n + j1) * R_l + k) * rmax + a0;
      const T* q2 = Qp + sL + ((long long)j2 * R_l + k) * rmax + b0;
      const T* q3 = Qp + 2 * sL + ((long long)j3 * R_l + k) * rmax + c0;
      for (int q = part; q < 32; q += 8) sA[kk][q] = (ok && a0 + q < rmax) ? q1[q] : T(0);
      sB[kk][part] = (ok && b0 + part < rmax) ? z * q2[part] : T(0);
      sC[kk][part] = (ok && c0 + part < rmax) ? q3[part] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      T ab = sA[kk][a] * sB[kk][bl];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = fma(ab, sC[kk][q], acc[q]);
    }
    __syncthreads();
    if (++chunk_count == 2) {
#pragma unroll
      for (int q = 0; q < 8; ++q) { acc64[q] += (double)acc[q]; acc[q] = T(0); }
      chunk_count = 0;
    }
  }
  const int aa = a0 + a, bb = b0 + bl;
  if (aa < r1 && bb < r2) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int cc = c0 + q;
      if (cc < r3) atomicAdd(&beta64[((long long)aa * rmax + bb) * rmax + cc], acc64[q] + (double)acc[q]);
    }
  }
}

// beta in the bulk type, and ||beta[a, :, :]||^2 per slice a (block partial sums in shared
// memory, one global atomic per slice and block)
template <typename T>
__global__ void convert_beta_kernel(const double* beta64, T* beta, long long tot, int rmax,
                                    DevScalars* sc) {
  __shared__ double acc[RMAX_LIMIT];
  for (int a = threadIdx.x; a < rmax; a += blockDim.x) acc[a] = 0.0;
  __syncthreads();
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < tot) {
    const double v = beta64[e];
    beta[e] = (T)v;
    if (v != 0.0) atomicAdd(&acc[e / ((long long)rmax * rmax)], v * v);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < rmax; a += blockDim.x)
    if (acc[a] != 0.0) atomicAdd(&sc->beta_a2[a], acc[a]);
}

// adims[a] = n for a < r_1 (batches of the mode-2 product that carry data), else 0;
// kdims[a] = r_2 (inner size of every batch)
__global__ void batch_dims_kernel(int* adims, int* kdims, int rmax, int n, const DevScalars* sc) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < rmax) {
    adims[a] = (a < sc->rank[0]) ? n : 0;
    kdims[a] = sc->rank[1];
  }
}

template <typename T>
static int projection_core_t(Ctx& c) {
  const int n = c.n, rmax = c.rmax;
  T* Qp = (T*)c.Qp;
  dim3 g1((n + 31) / 32, c.R_l, 3);
  proj_kernel<T><<<g1, 256, 0, c.stream>>>(Bulk<T>::Z(c), Bulk<T>::pk(c), n, rmax, c.R_l, c.sc, Qp);
  long long tot = (long long)rmax * rmax * rmax;
  cudaMemsetAsync(c.beta64, 0, sizeof(double) * tot, c.stream);
  const int ta = (rmax + 31) / 32, tb = (rmax + 7) / 8;
  // split K so that the whole GPU is busy even for small ranks
  int ksplit = 16;
  dim3 g2(ta * tb * tb, ksplit);
  core_kernel<T><<<g2, 256, 0, c.stream>>>(Qp, c.j, c.nz_idx, c.Z, n, rmax, c.R_l, c.sc, c.beta64);
  convert_beta_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(c.beta64, (T*)c.beta, tot,
                                                                                rmax, c.sc);
  // T1[a][b][i3] = sum_c beta[a][b][c] V3[i3][c]      (rows (a,b), K = r3)
  const T* Zb = Bulk<T>::Z(c);
  const long long sZ = (long long)n * rmax;
  gemm_batched<T>(c.stream, false, true, rmax * rmax, n, rmax, T(1), (const T*)c.beta, rmax, 0,
                  Zb + 2 * sZ, rmax, 0, T(0), (T*)c.T1, n, 0, 1, 1, nullptr, nullptr, c.sc->rank + 2);
  // T2[a][i2][i3] = sum_b V2[i2][b] T1[a][b][i3]        (batch a < r1, K = r2)
  if (c.use_tc && !c.fp64) return 4 + launch_t2_tiles(c);   // tiled FP16 operands
  batch_dims_kernel<<<(rmax + 127) / 128, 128, 0, c.stream>>>(c.adims, c.kdims, rmax, n, c.sc);
  gemm_batched<T>(c.stream, false, false, n, n, rmax, T(1), Zb + sZ, rmax, 0, (const T*)c.T1, n,
                  (long long)rmax * n, T(0), (T*)c.T2, c.t2_ld, (long long)n * c.t2_ld, rmax, 1,
                  c.adims, nullptr, c.kdims);
  return 6;
}

int launch_projection_core(Ctx& c) {
  return c.fp64 ? projection_core_t<double>(c) : projection_core_t<float>(c);
}

// ------------------------------------------------------------------ particle bins
__global__ void bin_count_kernel(const int* jidx, const int* nz_idx, const DevScalars* sc, int nb,
                                 int* count) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= sc->n_nz) return;
  int p = nz_idx[m];
  int b = ((jidx[3 * p] / BIN) * nb + jidx[3 * p + 1] / BIN) * nb + jidx[3 * p + 2] / BIN;
  atomicAdd(&count[b], 1);
}

__global__ void bin_scan_kernel(const int* count, int nbins, int* start) {
  __shared__ int scan[1024];
  const int T = blockDim.x, t = threadIdx.x;
  const int per = (nbins + T - 1) / T;
  const int b0 = min(nbins, t * per), b1 = min(nbins, b0 + per);
  int s = 0;
  for (int b = b0; b < b1; ++b) s += count[b];
  scan[t] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    int v = (t >= o) ? scan[t - o] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int pos = scan[t] - s;
  for (int b = b0; b < b1; ++b) { start[b] = pos; pos += count[b]; }
  if (t == T - 1) start[nbins] = scan[t];
}

__global__ void bin_fill_kernel(const int* jidx, const int* nz_idx, const DevScalars* sc, int nb,
                                const int* start, int* cursor, int* items) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= sc->n_nz) return;
  int p = nz_idx[m];
  int b = ((jidx[3 * p] / BIN) * nb + jidx[3 * p + 1] / BIN) * nb + jidx[3 * p + 2] / BIN;
  int pos = atomicAdd(&cursor[b], 1);
  items[start[b] + pos] = p;
}

// make each bin's order deterministic (ascending particle index)
__global__ void bin_sort_kernel(const int* start, int nbins, int* items) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  int s = start[b], e = start[b + 1];
  for (int i = s + 1; i < e; ++i) {
    int v = items[i], q = i - 1;
    while (q >= s && items[q] > v) { items[q + 1] = items[q]; --q; }
    items[q + 1] = v;
  }
}

int launch_bins(Ctx& c) {
  const int nb = c.nbin, nbins = nb * nb * nb;
  cudaMemsetAsync(c.bin_count, 0, sizeof(int) * (nbins + 1), c.stream);
  int grid = (c.maxN + 255) / 256;
  if (grid < 1) grid = 1;
  bin_count_kernel<<<grid, 256, 0, c.stream>>>(c.j, c.nz_idx, c.sc, nb, c.bin_count);
  bin_scan_kernel<<<1, 1024, 0, c.stream>>>(c.bin_count, nbins, c.bin_start);
  cudaMemsetAsync(c.bin_count, 0, sizeof(int) * (nbins + 1), c.stream);
  bin_fill_kernel<<<grid, 256, 0, c.stream>>>(c.j, c.nz_idx, c.sc, nb, c.bin_start, c.bin_count,
                                              c.bin_items);
  bin_sort_kernel<<<(nbins + 255) / 256, 256, 0, c.stream>>>(c.bin_start, nbins, c.bin_items);
  int k = 4;
  if (c.use_tc) k += launch_window_lists(c);
  return k;
}

// ------------------------------------------------------------------ windows (a6)
// Adds sum_{nu in L(i)} z_nu sum_{k short} p_k[i1-j1] p_k[i2-j2] p_k[i3-j3] over |i_l - j_l| <= gamma
// to the output (the cumulated canonical tensor of Defs. 3.4 and 3.6; overlapping windows add,
// Example 3.5).  Gather form: each CTA owns an 8 x 16 x 64 tile, collects the windows that
// reach it from the particle bins, sorts them (fixed summation order), stages their factor
// slices in shared memory in batches and adds them to the tile in one read-modify-write.
constexpr int WT1 = 8, WT2 = 16, WT3 = 64, WRS = 16, WMAXC = 256, WBATCH = 4, WTHREADS = 512;
template <typename T>
__global__ void __launch_bounds__(WTHREADS)
windows_kernel(T* P, const T* __restrict__ pk, const int* __restrict__ jidx, const double* __restrict__ Z,
               const int* __restrict__ bstart, const int* __restrict__ items, int n, int R, int R_l,
               int nb, DevScalars* sc) {
  const int nt3 = (n + WT3 - 1) / WT3, nt2 = (n + WT2 - 1) / WT2;
  int bt = blockIdx.x;
  const int t3 = bt % nt3; bt /= nt3;
  const int t2 = bt % nt2; bt /= nt2;
  const int t1 = bt;
  const int lo1 = t1 * WT1, lo2 = t2 * WT2, lo3 = t3 * WT3;
  const int hi1 = min(n, lo1 + WT1) - 1, hi2 = min(n, lo2 + WT2) - 1, hi3 = min(n, lo3 + WT3) - 1;
  const int g = sc->gamma;
  const int R_s = R - R_l;
  const int L = 2 * n - 1;
  const int b1a = max(0, lo1 - g) / BIN, b1b = min(n - 1, hi1 + g) / BIN;
  const int b2a = max(0, lo2 - g) / BIN, b2b = min(n - 1, hi2 + g) / BIN;
  const int b3a = max(0, lo3 - g) / BIN, b3b = min(n - 1, hi3 + g) / BIN;
  const int nb3 = b3b - b3a + 1, nb2 = b2b - b2a + 1, nbt = (b1b - b1a + 1) * nb2 * nb3;
  __shared__ int cand[WMAXC];
  __shared__ int s_total, s_cnt;
  __shared__ T g1[WBATCH][WRS][WT1];
  __shared__ T f2[WBATCH][WRS][WT2];
  __shared__ T f3[WBATCH][WRS][WT3];
  __shared__ int win[WBATCH][6];
  const int tid = threadIdx.x;
  const int i3o = tid % WT3, rg = tid / WT3;        // rows rg, rg+8, ..., rg+120 of the 128 (i1,i2) rows
  T acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = T(0);

  auto collect = [&](int rounds, int r) {
    if (tid == 0) { s_total = 0; s_cnt = 0; }
    __syncthreads();
    for (int t = tid; t < nbt; t += WTHREADS) {
      int b3 = b3a + t % nb3, b2 = b2a + (t / nb3) % nb2, b1 = b1a + t / (nb3 * nb2);
      int b = (b1 * nb + b2) * nb + b3;
      for (int it = bstart[b]; it < bstart[b + 1]; ++it) {
        int p = items[it];
        int j1 = jidx[3 * p], j2 = jidx[3 * p + 1], j3 = jidx[3 * p + 2];
        if (j1 < lo1 - g || j1 > hi1 + g || j2 < lo2 - g || j2 > hi2 + g || j3 < lo3 - g || j3 > hi3 + g)
          continue;
        atomicAdd(&s_total, 1);
        if (rounds > 1 && (p % rounds) != r) continue;
        int pos = atomicAdd(&s_cnt, 1);
        if (pos < WMAXC) cand[pos] = p;
      }
    }
    __syncthreads();
  };
  auto sort_cand = [&](int nc) {              // bitonic sort of cand[0..nc) (ascending)
    int m = 1;
    while (m < nc) m <<= 1;
    for (int i = nc + tid; i < m; i += WTHREADS) cand[i] = 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
      for (int jx = k >> 1; jx > 0; jx >>= 1) {
        for (int i = tid; i < m; i += WTHREADS) {
          int ixj = i ^ jx;
          if (ixj > i) {
            int a = cand[i], b = cand[ixj];
            bool up = (i & k) == 0;
            if ((a > b) == up) { cand[i] = b; cand[ixj] = a; }
          }
        }
        __syncthreads();
      }
  };
  auto process = [&](int nc) {
    for (int c0 = 0; c0 < nc; c0 += WBATCH) {
      const int nbat = min(WBATCH, nc - c0);
      for (int e = tid; e < nbat * R_s * (WT1 + WT2 + WT3); e += WTHREADS) {
        int cI = e / (R_s * (WT1 + WT2 + WT3));
        int rem = e % (R_s * (WT1 + WT2 + WT3));
        int k = rem / (WT1 + WT2 + WT3), o = rem % (WT1 + WT2 + WT3);
        int p = cand[c0 + cI];
        const T* rowk = pk + (long long)(R_l + k) * L + (n - 1);
        if (o < WT1) {
          int i = lo1 + o, d = i - jidx[3 * p];
          g1[cI][k][o] = (i < n && d >= -g && d <= g) ? (T)Z[p] * rowk[d] : T(0);
        } else if (o < WT1 + WT2) {
          int i = lo2 + o - WT1, d = i - jidx[3 * p + 1];
          f2[cI][k][o - WT1] = (i < n && d >= -g && d <= g) ? rowk[d] : T(0);
        } else {
          int i = lo3 + o - WT1 - WT2, d = i - jidx[3 * p + 2];
          f3[cI][k][o - WT1 - WT2] = (i < n && d >= -g && d <= g) ? rowk[d] : T(0);
        }
      }
      if (tid < nbat) {
        int p = cand[c0 + tid];
        win[tid][0] = max(0, jidx[3 * p] - g - lo1);     win[tid][1] = min(WT1 - 1, jidx[3 * p] + g - lo1);
        win[tid][2] = max(0, jidx[3 * p + 1] - g - lo2); win[tid][3] = min(WT2 - 1, jidx[3 * p + 1] + g - lo2);
        win[tid][4] = max(0, jidx[3 * p + 2] - g - lo3); win[tid][5] = min(WT3 - 1, jidx[3 * p + 2] + g - lo3);
      }
      __syncthreads();
      for (int cI = 0; cI < nbat; ++cI) {
        if (i3o < win[cI][4] || i3o > win[cI][5]) continue;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int rr = rg + 8 * q, i1o = rr / WT2, i2o = rr % WT2;
          if (i1o < win[cI][0] || i1o > win[cI][1] || i2o < win[cI][2] || i2o > win[cI][3]) continue;
          T v = T(0);
          for (int k = 0; k < R_s; ++k) v = fma(g1[cI][k][i1o] * f2[cI][k][i2o], f3[cI][k][i3o], v);
          acc[q] += v;
        }
      }
      __syncthreads();
    }
  };

  collect(1, 0);
  const int total = s_total;
  if (total == 0) return;                        // uniform: no window reaches this tile
  int rounds = 1;
  if (total > WMAXC) rounds = (total + WMAXC / 2 - 1) / (WMAXC / 2);
  for (int r = 0; r < rounds; ++r) {
    if (rounds > 1) collect(rounds, r);
    int nc = s_cnt;
    if (nc > WMAXC) {                            // pathological crowding: report, keep what fits
      if (tid == 0) atomicOr(&sc->flags, (unsigned)FLAG_WINDOWS);
      nc = WMAXC;
    }
    sort_cand(nc);
    process(nc);
  }
  const int i3 = lo3 + i3o;
  if (i3 >= n) return;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int rr = rg + 8 * q;
    const int i1 = lo1 + rr / WT2, i2 = lo2 + rr % WT2;
    if (i1 < n && i2 < n) {
      T* o = P + ((long long)i1 * n + i2) * n + i3;
      *o += acc[q];
    }
  }
}

template <typename T>
static int recon_gemm_t(Ctx& c, T* out) {
  const int n = c.n, rmax = c.rmax;
  const T* Zb = Bulk<T>::Z(c);
  if (c.t2_ld == n) {
    // P[i1][(i2,i3)] = sum_a V1[i1][a] T2[a][(i2,i3)]
    gemm_batched<T>(c.stream, false, false, n, n * n, rmax, T(1), Zb, rmax, 0, (const T*)c.T2,
                    n * n, 0, T(0), out, n * n, 0, 1, 1, nullptr, nullptr, c.sc->rank + 0);
  } else {
    // padded T2 rows: one batch per i2, P[i1][i2][i3] = sum_a V1[i1][a] T2[a][i2][i3]
    const long long ldb = (long long)n * c.t2_ld;
    gemm_batched<T>(c.stream, false, false, n, n, rmax, T(1), Zb, rmax, 0, (const T*)c.T2,
                    (int)ldb, c.t2_ld, T(0), out, n * n, n, n, 1, nullptr, nullptr,
                    c.sc->rank + 0);
  }
  return 1;
}

template <typename T>
static int windows_t(Ctx& c, T* out) {
  const int n = c.n;
  const int nt = ((n + WT1 - 1) / WT1) * ((n + WT2 - 1) / WT2) * ((n + WT3 - 1) / WT3);
  windows_kernel<T><<<nt, WTHREADS, 0, c.stream>>>(out, Bulk<T>::pk(c), c.j, c.Z, c.bin_start,
                                                   c.bin_items, n, c.R, c.R_l, c.nbin, c.sc);
  return 1;
}

int launch_recon_gemm(Ctx& c, void* out) {
  if (c.fp64) return recon_gemm_t<double>(c, (double*)out);
  // FP32 bulk: the tensor-core assembly (Tucker product and windows in one kernel) when the
  // context planned it, else the CUDA-core product followed by the window kernel
  if (c.use_tc) return launch_assemble(c, (float*)out);
  return recon_gemm_t<float>(c, (float*)out);
}

int launch_windows(Ctx& c, void* out) {
  if (!c.fp64 && c.use_tc) return 0;      // the tensor-core assembly already added the windows
  return c.fp64 ? windows_t<double>(c, (double*)out) : windows_t<float>(c, (float*)out);
}

// ------------------------------------------------------------------ point evaluation, energy
// A(i) = sum_{a,b} V1[i1][a] V2[i2][b] T1[a][b][i3]  +  sum_{nu in L(i)} z_nu U_nu(i)   (Lemma 3.10)
template <typename T>
__device__ double rs_point_value(const DevView& c, const T* Zb, const T* T1, int i1, int i2, int i3,
                                 int lane) {
  const int n = c.n, rmax = c.rmax;
  const int r1 = c.sc->rank[0], r2 = c.sc->rank[1];
  const long long sZ = (long long)n * rmax;
  double v = 0.0;
  for (int e = lane; e < r1 * r2; e += 32) {
    int a = e / r2, b = e % r2;
    double t1 = (double)T1[((long long)a * rmax + b) * n + i3];
    v += (double)Zb[(long long)i1 * rmax + a] * (double)Zb[sZ + (long long)i2 * rmax + b] * t1;
  }
  // short-range windows (FP64 factors)
  const int g = c.sc->gamma, L = 2 * n - 1, nb = c.nbin;
  const int b1a = max(0, i1 - g) / BIN, b1b = min(n - 1, i1 + g) / BIN;
  const int b2a = max(0, i2 - g) / BIN, b2b = min(n - 1, i2 + g) / BIN;
  const int b3a = max(0, i3 - g) / BIN, b3b = min(n - 1, i3 + g) / BIN;
  const int nb3 = b3b - b3a + 1, nb2 = b2b - b2a + 1;
  const int nbt = (b1b - b1a + 1) * nb2 * nb3;
  for (int t = lane; t < nbt; t += 32) {
    int b3 = b3a + t % nb3, b2 = b2a + (t / nb3) % nb2, b1 = b1a + t / (nb3 * nb2);
    int b = (b1 * nb + b2) * nb + b3;
    for (int it = c.bin_start[b]; it < c.bin_start[b + 1]; ++it) {
      int p = c.bin_items[it];
      int d1 = i1 - c.j[3 * p], d2 = i2 - c.j[3 * p + 1], d3 = i3 - c.j[3 * p + 2];
      if (abs(d1) > g || abs(d2) > g || abs(d3) > g) continue;
      double s = 0.0;
      for (int k = c.R_l; k < c.R; ++k) {
        const double* row = c.pk64 + (long long)k * L + n - 1;
        s += row[d1] * row[d2] * row[d3];
      }
      v += c.Z[p] * s;
    }
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;     // valid in lane 0
}

template <typename T>
__global__ void energy_kernel(DevView c, const T* Zb, const T* T1, double* part) {
  __shared__ double red[8];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m = blockIdx.x * 8 + warp;
  double e = 0.0;
  if (m < c.sc->n_nz) {
    int p = c.nz_idx[m];
    double A = rs_point_value<T>(c, Zb, T1, c.j[3 * p], c.j[3 * p + 1], c.j[3 * p + 2], lane);
    double z = c.Z[p];
    e = z * (A - z * c.sc->P_R0);
  }
  if (lane == 0) red[warp] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

__global__ void energy_sum_kernel(const double* part, int nparts, DevScalars* sc) {
  __shared__ double red[32];
  double s = 0.0;
  // fixed-order: thread t sums a contiguous chunk
  int per = (nparts + blockDim.x - 1) / blockDim.x;
  int b0 = min(nparts, (int)threadIdx.x * per), b1 = min(nparts, b0 + per);
  for (int i = b0; i < b1; ++i) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    sc->energy = 0.5 * t;
  }
}

template <typename T>
__global__ void eval_points_kernel(DevView c, const T* Zb, const T* T1, int M, const int* idx,
                                   double* out) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m = blockIdx.x * 8 + warp;
  if (m >= M) return;
  int i1 = min(max(idx[3 * m], 0), c.n - 1), i2 = min(max(idx[3 * m + 1], 0), c.n - 1),
      i3 = min(max(idx[3 * m + 2], 0), c.n - 1);
  double v = rs_point_value<T>(c, Zb, T1, i1, i2, i3, lane);
  if (lane == 0) out[m] = v;
}

int launch_energy(Ctx& c, int N) {
  int blocks = (c.maxN + 7) / 8;
  if (blocks < 1) blocks = 1;
  DevView v = make_view(c);
  if (c.fp64) energy_kernel<double><<<blocks, 256, 0, c.stream>>>(v, c.Z64, (const double*)c.T1, c.Epart);
  else energy_kernel<float><<<blocks, 256, 0, c.stream>>>(v, c.Z32, (const float*)c.T1, c.Epart);
  energy_sum_kernel<<<1, 1024, 0, c.stream>>>(c.Epart, blocks, c.sc);
  (void)N;
  return 2;
}

int launch_eval_points(Ctx& c, int M, const int* idx, double* out) {
  if (M <= 0) return 0;
  int blocks = (M + 7) / 8;
  DevView v = make_view(c);
  if (c.fp64) eval_points_kernel<double><<<blocks, 256, 0, c.stream>>>(v, c.Z64, (const double*)c.T1, M, idx, out);
  else eval_points_kernel<float><<<blocks, 256, 0, c.stream>>>(v, c.Z32, (const float*)c.T1, M, idx, out);
  return 1;
}

}  // namespace rs
