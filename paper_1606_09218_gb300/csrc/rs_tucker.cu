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
// factors; the projected side matrix is U~^(l)[a, (nu,k)] = w_nu Qp[l][j_l^(nu)][k][a]).  Only the
// coordinates j that carry charge (the compacted list nzj) are computed; a >= r_l is zero.
// CTA: 64 rows j x 64 columns a for one (l, k); thread: 4 j x 4 a; K = i in chunks of 32 with
// the full factor row p_k in shared memory.
template <typename T>
__global__ void __launch_bounds__(256)
proj_kernel(const T* __restrict__ Zb, const T* __restrict__ pk, const int* __restrict__ nzj, int n,
            int rmax, int R_l, DevScalars* sc, T* Qp) {
  extern __shared__ __align__(16) unsigned char psm[];
  T* sp = (T*)psm;                                   // p_k[d], d = -(n-1) .. n-1
  T* sV = sp + ((2 * n - 1 + 3) & ~3);               // [32][64] slice of Z_l
  const int l = blockIdx.z, k = blockIdx.y;
  const int nat = (rmax + 63) / 64;
  const int j0 = (blockIdx.x / nat) * 64, a0 = (blockIdx.x % nat) * 64;
  const int cnt = sc->nzj_count[l], r = sc->rank[l];
  if (j0 >= cnt) return;
  const int L = 2 * n - 1;
  const int tid = threadIdx.x, tj = tid >> 4, ta = tid & 15;
  int jj[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int idx = j0 + 4 * tj + x;
    jj[x] = idx < cnt ? nzj[l * n + idx] : -1;
  }
  T acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
  if (a0 < r) {
    const T* pkk = pk + (long long)k * L;
    for (int e = tid; e < L; e += 256) sp[e] = pkk[e];
    const T* Zl = Zb + (long long)l * n * rmax;
    for (int i0 = 0; i0 < n; i0 += 32) {
      __syncthreads();
      for (int e = tid; e < 32 * 64; e += 256) {
        const int ii = e >> 6, aa = e & 63, i = i0 + ii, a = a0 + aa;
        sV[e] = (i < n && a < r) ? Zl[(long long)i * rmax + a] : T(0);
      }
      __syncthreads();
      const int ilim = min(32, n - i0);
      // factor rows p_k[i - j] of this thread's four j, as pointers advancing with i (a padding
      // row, jj < 0, reads the row of j = 0 and is never stored)
      const T* pr[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) pr[x] = sp + (i0 + n - 1) - max(jj[x], 0);
      for (int ii = 0; ii < ilim; ++ii) {
        T v[4], pj[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) v[y] = sV[ii * 64 + 4 * ta + y];
#pragma unroll
        for (int x = 0; x < 4; ++x) pj[x] = pr[x][ii];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(pj[x], v[y], acc[x][y]);
      }
    }
  }
  float qm = 0.f;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    if (jj[x] < 0) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int a = a0 + 4 * ta + y;
      if (a < rmax) Qp[(((long long)l * n + jj[x]) * R_l + k) * rmax + a] = (a < r) ? acc[x][y] : T(0);
      if (a < r) qm = fmaxf(qm, fabsf((float)acc[x][y]));
    }
  }
  // largest |Qp| (operand scale of the tensor-core core contraction)
  for (int o = 16; o > 0; o >>= 1) qm = fmaxf(qm, __shfl_xor_sync(0xffffffffu, qm, o));
  if ((threadIdx.x & 31) == 0 && qm > 0.f) atomicMax(&sc->qmax_bits, __float_as_uint(qm));
}

// ------------------------------------------------------------------ core
// beta[a][b][c] = sum_{p nonzero} z_p sum_{k long} Qp1[j1][k][a] Qp2[j2][k][b] Qp3[j3][k][c]
// (Eq. (6.2): beta = xi x_1 U~1 x_2 U~2 x_3 U~3 with xi = sign z and w^3 = |z|).
// CTA tile: 64 a x 4 b x 32 c over a slice of K = (particle, k); thread: 4 a x 1 b x 8 c.
// FP32 path: products in FP32, each 32-term chunk added to a (hi, lo) FP32 pair with an
// error-free two-sum, so the K sum carries about twice the FP32 precision; the CTA's partial
// sums are added to beta64 in FP64.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

constexpr int CORE_KMAX = 1024;           // K elements of one CTA (row offsets kept in shared memory)

template <typename T>
constexpr size_t core_smem_bytes() {
  return sizeof(T) * (2 * 32 * 100 + CORE_KMAX) + sizeof(int) * 3 * CORE_KMAX;
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool in) {
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(in ? 4 : 0) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(in ? 8 : 0) : "memory");
}

template <typename T>
__global__ void __launch_bounds__(256, 2)
core_kernel(const T* __restrict__ Qp, const int* __restrict__ jidx, const int* __restrict__ nz_idx,
            const double* __restrict__ Z, int n, int rmax, int R_l, const DevScalars* sc,
            double* beta64) {
  const int r1 = sc->rank[0], r2 = sc->rank[1], r3 = sc->rank[2];
  const int nbt = (rmax + 3) / 4, nct = (rmax + 31) / 32;
  int bt = blockIdx.x;
  const int cI = bt % nct; bt /= nct;
  const int bI = bt % nbt; bt /= nbt;
  const int a0 = bt * 64, b0 = bI * 4, c0 = cI * 32;
  if (a0 >= r1 || b0 >= r2 || c0 >= r3) return;
  const int nnz = sc->n_nz;
  const long long Ktot = (long long)nnz * R_l;
  const long long per = (Ktot + gridDim.y - 1) / gridDim.y;
  const long long kb = blockIdx.y * per, ke = min(Ktot, kb + per);
  if (kb >= ke) return;
  extern __shared__ __align__(16) unsigned char csm[];
  T (*s1)[32][64] = (T(*)[32][64])csm;                          // [2][32][64]
  T (*s2)[32][4] = (T(*)[32][4])(csm + sizeof(T) * 2 * 32 * 64);  // [2][32][4]
  T (*s3)[32][32] = (T(*)[32][32])(csm + sizeof(T) * 2 * 32 * 68);  // [2][32][32]
  T* zK = (T*)(csm + sizeof(T) * 2 * 32 * 100);                 // [CORE_KMAX]
  int* off1 = (int*)(csm + sizeof(T) * (2 * 32 * 100 + CORE_KMAX));
  int* off2 = off1 + CORE_KMAX;
  int* off3 = off2 + CORE_KMAX;
  __shared__ T zs[32][4];                         // z_K q2[K][b] of the current chunk
  const int tid = threadIdx.x;
  const int nK = (int)(ke - kb);                  // <= CORE_KMAX (host sizes the split)
  const long long sL = (long long)n * R_l * rmax;
  // row offsets of the three projected factors and the charge, for every K of this CTA
  for (int e = tid; e < nK; e += 256) {
    const long long K = kb + e;
    const int p = nz_idx[K / R_l], k = (int)(K % R_l);
    off1[e] = (int)(((long long)jidx[3 * p] * R_l + k) * rmax);
    off2[e] = (int)(sL + ((long long)jidx[3 * p + 1] * R_l + k) * rmax);
    off3[e] = (int)(2 * sL + ((long long)jidx[3 * p + 2] * R_l + k) * rmax);
    zK[e] = (T)Z[p];
  }
  __syncthreads();
  // gathers of one chunk of 32 K into buffer bf (zero outside K range / ranks)
  auto stage = [&](int ch, int bf) {
    for (int e = tid; e < 32 * 100; e += 256) {
      const int kk = e / 100, part = e - kk * 100;
      const int kl = ch * 32 + kk;
      const bool ok = kl < nK;
      if (part < 64) {
        const int a = a0 + part;
        cp_async_elem(&s1[bf][kk][part], Qp + (ok ? off1[kl] + a : 0), ok && a < rmax);
      } else if (part < 68) {
        const int b = b0 + part - 64;
        cp_async_elem(&s2[bf][kk][part - 64], Qp + (ok ? off2[kl] + b : 0), ok && b < rmax);
      } else {
        const int c = c0 + part - 68;
        cp_async_elem(&s3[bf][kk][part - 68], Qp + (ok ? off3[kl] + c : 0), ok && c < rmax);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int ta = tid & 15, tb = (tid >> 4) & 3, tc = tid >> 6;    // 4 a x 1 b x 8 c per thread
  T acc[4][8];
  T hi[4][8], lo[4][8];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 8; ++y) { acc[x][y] = T(0); hi[x][y] = T(0); lo[x][y] = T(0); }
  const int nch = (nK + 31) / 32;
  stage(0, 0);
  for (int ch = 0; ch < nch; ++ch) {
    const int bf = ch & 1;
    if (ch + 1 < nch) {
      stage(ch + 1, bf ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    // z_K q2[K][b] of the chunk, once per (K, b) instead of once per thread
    if (tid < 128) {
      const int kk = tid >> 2, bq = tid & 3, kl = ch * 32 + kk;
      zs[kk][bq] = (kl < nK ? zK[kl] : T(0)) * s2[bf][kk][bq];
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      const T zb = zs[kk][tb];
      T t[4], q3[8];
#pragma unroll
      for (int x = 0; x < 4; ++x) t[x] = s1[bf][kk][4 * ta + x] * zb;
#pragma unroll
      for (int y = 0; y < 8; ++y) q3[y] = s3[bf][kk][8 * tc + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fma(t[x], q3[y], acc[x][y]);
    }
    // fold the chunk sum into the (hi, lo) pair
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        if (sizeof(T) == 4) two_sum_add(*(float*)&hi[x][y], *(float*)&lo[x][y], (float)acc[x][y]);
        else hi[x][y] += acc[x][y];
        acc[x][y] = T(0);
      }
    __syncthreads();                              // buffer bf is refilled two chunks later
  }
  const int bb = b0 + tb;
  if (bb >= r2) return;
  const double pfx = ldexp(1.0, beta_fx_shift(sc, R_l));
  unsigned long long* bfx = reinterpret_cast<unsigned long long*>(beta64);
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int aa = a0 + 4 * ta + x;
    if (aa >= r1) continue;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const int cc = c0 + 8 * tc + y;
      if (cc < r3)
        atomicAdd(&bfx[((long long)aa * rmax + bb) * rmax + cc], beta_fx((double)hi[x][y] + (double)lo[x][y], pfx));
    }
  }
}

// beta from its fixed-point sums (in place as FP64, and in the bulk type), and ||beta[a, :, :]||^2
// per slice a (one CTA per slice)
template <typename T>
__global__ void __launch_bounds__(256)
convert_beta_kernel(double* beta64, T* beta, int rmax, int R_l, DevScalars* sc) {
  __shared__ double red[8];
  const int a = blockIdx.x;
  const long long base = (long long)a * rmax * rmax;
  const double pinv = ldexp(1.0, -beta_fx_shift(sc, R_l));
  long long* bfx = reinterpret_cast<long long*>(beta64);
  double s = 0.0;
  for (int e = threadIdx.x; e < rmax * rmax; e += blockDim.x) {
    const double v = (double)bfx[base + e] * pinv;
    beta64[base + e] = v;
    beta[base + e] = (T)v;
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    sc->beta_a2[a] = t;
  }
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
  const size_t psmem = sizeof(T) * ((size_t)((2 * n - 1 + 3) & ~3) + 32 * 64);
  dim3 g1(((n + 63) / 64) * ((rmax + 63) / 64), c.R_l, 3);
  proj_kernel<T><<<g1, 256, psmem, c.stream>>>(Bulk<T>::Z(c), Bulk<T>::pk(c), c.nzj, n, rmax, c.R_l, c.sc, Qp);
  long long tot = (long long)rmax * rmax * rmax;
  cudaMemsetAsync(c.beta64, 0, sizeof(double) * tot, c.stream);
  // split K so that the whole GPU is busy even for small ranks
  const int ntile = ((rmax + 63) / 64) * ((rmax + 3) / 4) * ((rmax + 31) / 32);
  int ksplit = (8 * 152 + ntile - 1) / ntile;
  if (ksplit < 1) ksplit = 1;
  // every CTA keeps the row offsets of its K range in shared memory
  const long long kmax = (long long)c.maxN * c.R_l;
  const int kmin_split = (int)((kmax + CORE_KMAX - 1) / CORE_KMAX);
  if (ksplit < kmin_split) ksplit = kmin_split;
  dim3 g2(ntile, ksplit);
  int kcore = 1;
  if (sizeof(T) == 4 && c.use_kr_core)
    kcore = launch_core_kr(c);                       // tcgen05, Khatri-Rao operands formed once
  else if (sizeof(T) == 4 && c.use_tc_core)
    kcore = launch_core_tc(c);                       // tcgen05, FP16-split operands
  else
    core_kernel<T><<<g2, 256, core_smem_bytes<T>(), c.stream>>>(Qp, c.j, c.nz_idx, c.Z, n, rmax, c.R_l, c.sc,
                                                                 c.beta64);
  convert_beta_kernel<T><<<rmax, 256, 0, c.stream>>>(c.beta64, (T*)c.beta, rmax, c.R_l, c.sc);
  // T1[a][b][i3] = sum_c beta[a][b][c] V3[i3][c]      (rows (a,b), K = r3)
  const T* Zb = Bulk<T>::Z(c);
  const long long sZ = (long long)n * rmax;
  gemm_batched<T>(c.stream, false, true, rmax * rmax, n, rmax, T(1), (const T*)c.beta, rmax, 0,
                  Zb + 2 * sZ, rmax, 0, T(0), (T*)c.T1, n, 0, 1, nullptr, nullptr, c.sc->rank + 2, &c.gscr);
  // T2[a][i2][i3] = sum_b V2[i2][b] T1[a][b][i3]        (batch a < r1, K = r2)
  if (c.use_tc && !c.fp64) return 3 + kcore + launch_t2_tiles(c);   // tiled FP16 operands
  batch_dims_kernel<<<(rmax + 127) / 128, 128, 0, c.stream>>>(c.adims, c.kdims, rmax, n, c.sc);
  gemm_batched<T>(c.stream, false, false, n, n, rmax, T(1), Zb + sZ, rmax, 0, (const T*)c.T1, n,
                  (long long)rmax * n, T(0), (T*)c.T2, c.t2_ld, (long long)n * c.t2_ld, rmax,
                  c.adims, nullptr, c.kdims, &c.gscr);
  return 5 + kcore;
}

int launch_projection_core(Ctx& c) {
  return c.fp64 ? projection_core_t<double>(c) : projection_core_t<float>(c);
}

// FP64 projections of all three modes onto the FP64 bases (any precision of the context): the
// input of the ALS mode matrices.  Same layout as Qp; rows of uncharged coordinates untouched.
int launch_proj64(Ctx& c, double* Qp) {
  const int n = c.n, rmax = c.rmax;
  const size_t psmem = sizeof(double) * ((size_t)((2 * n - 1 + 3) & ~3) + 32 * 64);
  dim3 g1(((n + 63) / 64) * ((rmax + 63) / 64), c.R_l, 3);
  proj_kernel<double><<<g1, 256, psmem, c.stream>>>(c.Z64, c.pk64, c.nzj, n, rmax, c.R_l, c.sc, Qp);
  return 1;
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
                    n * n, 0, T(0), out, n * n, 0, 1, nullptr, nullptr, c.sc->rank + 0, &c.gscr);
  } else {
    // padded T2 rows: one batch per i2, P[i1][i2][i3] = sum_a V1[i1][a] T2[a][i2][i3]
    const long long ldb = (long long)n * c.t2_ld;
    gemm_batched<T>(c.stream, false, false, n, n, rmax, T(1), Zb, rmax, 0, (const T*)c.T2,
                    (int)ldb, c.t2_ld, T(0), out, n * n, n, n, nullptr, nullptr,
                    c.sc->rank + 0, &c.gscr);
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
  window_add(c, i1, i2, i3, lane, v);      // short-range windows (FP64 factors)
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
  else if (c.use_tc) launch_energy_t2(c, c.Epart, blocks);        // Tucker value from the T2 tiles
  else energy_kernel<float><<<blocks, 256, 0, c.stream>>>(v, c.Z32, (const float*)c.T1, c.Epart);
  energy_sum_kernel<<<1, 1024, 0, c.stream>>>(c.Epart, blocks, c.sc);
  (void)N;
  return 2;
}

// ------------------------------------------------------------------ forces (a9)
// F_j = -z_j [grad P_l(x_j) + sum_{nu in windows} z_nu grad U_nu(x_j)]  (Sec. 4.3).  The long
// part is the untruncated pair kernel,
//   grad P_l(x_j) = sum_{nu != j} z_nu sum_{k long} grad (p_k (x) p_k (x) p_k)(x_j - x_nu),
// exact for P_l by symmetry and O(eps) from the gradient of the RS-Tucker tensor; it has no
// division by the eigenvalues of the Gram matrices, which makes a continuation of the Tucker
// basis off the grid ill-conditioned for its weakest retained directions.  Factors and products
// in T (FP64 on the plain path, FP32 on the bulk path), sums in FP64.  The windows use the FP64
// factor and derivative tables; the self window contributes zero, since p_k' is odd.
// One warp per charged particle.
template <typename T>
__global__ void forces_direct_kernel(DevView c, const T* __restrict__ pk, const T* __restrict__ dpk,
                                     const double* __restrict__ dpk64, double* Fout) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m = blockIdx.x * 8 + warp;
  const int nnz = c.sc->n_nz;
  if (m >= nnz) return;
  const int p = c.nz_idx[m];
  const int n = c.n, L = 2 * n - 1;
  const int i1 = c.j[3 * p], i2 = c.j[3 * p + 1], i3 = c.j[3 * p + 2];
  double g1 = 0.0, g2 = 0.0, g3 = 0.0;
  for (int mm = lane; mm < nnz; mm += 32) {
    const int q = c.nz_idx[mm];
    if (q == p) continue;
    const int d1 = i1 - c.j[3 * q] + n - 1, d2 = i2 - c.j[3 * q + 1] + n - 1, d3 = i3 - c.j[3 * q + 2] + n - 1;
    T s1 = T(0), s2 = T(0), s3 = T(0);
    for (int k = 0; k < c.R_l; ++k) {
      const T* row = pk + (long long)k * L;
      const T* drow = dpk + (long long)k * L;
      const T f1 = row[d1], f2 = row[d2], f3 = row[d3];
      s1 = fma(drow[d1], f2 * f3, s1);
      s2 = fma(f1 * drow[d2], f3, s2);
      s3 = fma(f1 * f2, drow[d3], s3);
    }
    const double zq = c.Z[q];
    g1 += zq * (double)s1;
    g2 += zq * (double)s2;
    g3 += zq * (double)s3;
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

int launch_forces(Ctx& c) {
  cudaMemsetAsync(c.Fout, 0, sizeof(double) * 3 * (size_t)c.maxN, c.stream);
  int blocks = (c.maxN + 7) / 8;
  if (blocks < 1) blocks = 1;
  if (c.fp64)
    forces_direct_kernel<double><<<blocks, 256, 0, c.stream>>>(make_view(c), c.pk64, c.dpk64, c.dpk64, c.Fout);
  else
    forces_direct_kernel<float><<<blocks, 256, 0, c.stream>>>(make_view(c), c.pk32, c.dpk32, c.dpk64, c.Fout);
  return 1;
}

int launch_eval_points(Ctx& c, int M, const int* idx, double* out) {
  if (M <= 0) return 0;
  int blocks = (M + 7) / 8;
  DevView v = make_view(c);
  if (c.fp64) eval_points_kernel<double><<<blocks, 256, 0, c.stream>>>(v, c.Z64, (const double*)c.T1, M, idx, out);
  else eval_points_kernel<float><<<blocks, 256, 0, c.stream>>>(v, c.Z32, (const float*)c.T1, M, idx, out);
  return 1;
}

cudaError_t set_attributes_tucker(int optin) {
  cudaError_t e = allow_max_dynamic_smem((const void*)proj_kernel<float>, optin);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)proj_kernel<double>, optin);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)core_kernel<float>, optin);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)core_kernel<double>, optin);
  return e;
}

}  // namespace rs
