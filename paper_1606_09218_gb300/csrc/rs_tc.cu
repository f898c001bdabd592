// Tensor-core (tcgen05) assembly of the FP32 RS potential on the grid.  One GEMM per output
// tile with a data-dependent K:
//
//   P[i1][i2][i3] = sum_a V1[i1][a] T2[a][i2][i3]                        Tucker part (Def. 3.9,
//                                                                         Eq. (3.11); Eq. (2.3))
//                 + sum_{nu in L(i)} sum_{k short} (z_nu p_k[i2-j2] p_k[i3-j3]) p_k[i1-j1]
//                                                                         windows (Defs. 3.4, 3.6)
//
// M = 128 consecutive grid points p = i2 n + i3 of a plane, N = a chunk of i1 rows, K = the
// Tucker rank r1, then ceil8(R_s) per window that reaches the tile (a window is a rank-R_s outer
// product: one more K slice).  The sums live in tensor memory, the output is stored once and
// never read back: the Tucker product and the short-range windows cost one pass over the grid.
//
// Operands and precision (every operand x is split as x = hi + lo in FP16, |x - hi - lo| <=
// 2^-22 |x| in the normal range, and hi*hi + hi*lo + lo*hi accumulate in FP32):
//  * Tucker part (kind::f16, its own accumulator): T2 is written by the mode-2 product directly
//    as FP16 hi / lo tiles in the canonical K-major layout (one contiguous block per tile,
//    fetched with one bulk copy); V1 (|V1| <= 1) is scaled by 2^8 and T2 by 2^(S-8) with
//    2^(S-8) max_a ||beta[a]|| < 2^14, a bound of every T2 entry (|T2[a][i2][i3]| <=
//    ||beta[a,:,:]|| for orthonormal V2, V3): nothing overflows, and values below the FP16
//    normal range carry absolute errors far below the FP32 rounding of the result;
//  * windows (kind::f16, a second accumulator, scale 2^(sA+sB)): two windows share one K = 16
//    MMA (one 8-wide K chunk each); A_w[m][k] = 2^sA z p_k[i2-j2] p_k[i3-j3] is built per window,
//    while B = 2^sB p_k[i1-j1] is a slice of one factor table stored with a 16-byte row pitch,
//    so every row offset is a valid operand start and the two windows' slices are one leading
//    byte offset apart: no per-window B is built.
// The epilogue scales both accumulators back (exact powers of two) and adds them.
//
// CTA (persistent, one per SM, 18 warps):
//   warp 0     tensor-memory owner; lane 0 issues the MMAs (straight-line, descriptors precomputed)
//   warp 1     scheduler: bulk copy of the T2 tiles of the next jobs, window list pages
//   warps 2-9  producers, two groups of four: window operand pairs -> ring of slots (+ ready-made
//              descriptors); group g builds the pairs of parity g, so two pairs are built at once
//   warps 10-17 epilogue: tensor memory -> registers -> global, each warp writing 128-byte
//              runs of a plane row (streaming stores)
// A CTA keeps one i1 chunk (its V1 rows, split, as the B operand of the Tucker part) and walks
// over the tiles; the CTAs are spread over the chunks in proportion to their work (tiles plus
// windows).  Both accumulators are double-buffered so that the stores of one tile overlap the
// MMAs of the next.  Every wait is bounded: on expiry the CTA sets FLAG_TIMEOUT, the other roles
// see an abort flag, the MMA issuer and the copy issuers wait (bounded) for their work in
// flight, and the tensor memory is released before return.
#include "rs_internal.cuh"
#include "rs_tcgen05.cuh"

#include <cuda_fp16.h>

#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace rs {

namespace {

constexpr int AS_M = 128;                  // grid points per tile (tensor-memory lanes)
constexpr int AS_T3 = 32;                  // i3 columns per CTA of the T2 tile kernel
constexpr int AS_THREADS = 576;            // 18 warps
constexpr int WARP_SCHED = 1, WARP_PROD = 2, WARP_EPI = 10;
constexpr int NPW = 4;                     // warps of one producer group (one per operand row quarter)
constexpr int NPG = 2;                     // producer groups
constexpr int NEPI = 8;                    // epilogue warps
constexpr int NA_MAX = 3, NS_MAX = 8;      // T2 tile stages, window pair slots
constexpr int STG_ROW = 132;               // floats per staging row (128 + alignment shift)
constexpr int LIST_CAP = 256;              // window records per list page
constexpr int WL_SORT_CAP = 4096;          // longest window list of one tile column
constexpr int SMEM_LIMIT = 232448;         // opt-in shared memory per CTA on this GPU family
constexpr int SMEM_RESERVE = 1024;         // static shared memory of the kernel
constexpr double COST_TILE = 2500.0;       // relative cost of one tile job (output bound)
constexpr double COST_TILE_STAGED = 1500.0;  // ... with the staged epilogue (fitted: 1000 / 1500 / 2500
                                           // gave 492 / 416 / 424 us on the protein workload)
constexpr double COST_WINDOW = 87.0;       // relative cost of one window of a job (fitted to role traces:
                                           // about 7.8K cycles per job and 270 per window on the
                                           // protein workload, with two producer groups)
constexpr int TT_ROWS = 32;                // i2 rows per CTA of the T2 tile kernel

// Scale exponent S of the Tucker operands: 2^(S-8) max_a ||beta[a]|| < 2^14.
__device__ __forceinline__ int operand_shift(const DevScalars* sc, int r1) {
  double m = 0.0;
  for (int a = 0; a < r1; ++a) m = fmax(m, sc->beta_a2[a]);
  if (!(m > 0.0)) return 0;
  return max(-100, min(100, 22 - exp2_above(sqrt(m))));
}

struct AsmArgs {
  const unsigned char* T2t;   // FP16 hi / lo tiles of T2, tile_bytes each
  unsigned long long tile_bytes;
  const float* V1;            // mode-1 Tucker basis, n x ldv
  int ldv;
  const float* pk;            // factor table, R x L (FP32)
  const int4* rec;            // window records (j1, j2, j3, float bits of z), per tile
  const int2* rng;            // [tile][chunk] ranges into rec (nullptr: no short-range terms)
  float* P;                   // output n^3
  DevScalars* sc;
  int n, L, R_l, R_s;
  int nch, Nc, kp, gcap, TR, D0, ntiles, dstride, tmem_cols, na, ns;
  uint32_t off_bv, off_a, off_slot, off_tbl, off_tab, off_list, off_stage;
  int staged;                  // epilogue through shared staging rows and bulk stores
  double cost_tile;            // relative cost of a tile job in the CTA split (COST_TILE*)
  uint32_t bv_half, a_half, tbl_half;   // bytes of each hi part (the lo part follows)
};

constexpr uint32_t SLOT_HALF = AS_M * 16 * 2;    // one pair slot: 128 rows x K 16 FP16, hi or lo

}  // namespace

// ------------------------------------------------------------------ T2 tiles
// T2[a][i2][i3] = sum_b V2[i2][b] T1[a][b][i3]  (mode-2 product, Eq. (2.3)) written as the A
// operand of the assembly: per output tile (128 consecutive points p = i2 n + i3, K = kp ranks)
// an FP16 hi block and an FP16 lo block in the canonical K-major layout, scaled by 2^(S-8);
// ranks a >= r1 and points beyond the grid are zero.  One CTA: 32 i3 x 32 i2, ranks in stages
// of 4, two stages to a 16-byte chunk of a row.
__global__ void __launch_bounds__(256)
t2_tiles_kernel(const float* __restrict__ T1, const float* __restrict__ V2, int n, int rmax, int kp,
                int ntiles, DevScalars* sc, unsigned char* __restrict__ out,
                unsigned long long tile_bytes) {
  extern __shared__ __align__(16) float tsm[];
  float* T1s = tsm;                          // [2][rmax][32][4]: stage of ranks 4h + (0..3) at (b, i3)
  float* V2s = tsm + 8 * rmax * 32;          // [rmax][8][4]: V2[i2b + w + 8q][b] at (b, w, q)
  __shared__ float s_scale;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t3 = blockIdx.x, i2b = blockIdx.y * TT_ROWS, i3 = t3 * AS_T3 + lane;
  const int r1 = sc->rank[0], r2 = sc->rank[1];
  if (warp == 0) {
    // operand_shift(sc, r1), its maximum taken by one warp (the same exact maximum)
    double m = 0.0;
    for (int a = lane; a < r1; a += 32) m = fmax(m, sc->beta_a2[a]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      const int S = m > 0.0 ? max(-100, min(100, 22 - exp2_above(sqrt(m)))) : 0;
      s_scale = ldexpf(1.0f, S - 8);
      if (blockIdx.x == 0 && blockIdx.y == 0) sc->t2_shift = S;
    }
  }
  __syncthreads();
  const float scale = s_scale;
  const unsigned long long half_bytes = tile_bytes / 2;
  const long long np = (long long)n * n;
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    // rows of the last tile beyond the grid
    const long long p_last = (long long)(ntiles - 1) * AS_M;
    unsigned char* tile = out + (unsigned long long)(ntiles - 1) * tile_bytes;
    for (int e = tid; e < AS_M * (kp >> 3); e += 256) {
      const int m = e / (kp >> 3), k8 = e % (kp >> 3);
      if (p_last + m >= np) {
        const uint32_t off = kmajor_offset(m, k8, kp >> 3);
        *(uint4*)(tile + off) = make_uint4(0, 0, 0, 0);
        *(uint4*)(tile + half_bytes + off) = make_uint4(0, 0, 0, 0);
      }
    }
  }
  for (int r = warp; r < TT_ROWS; r += 8) {
    const int i2 = i2b + r;
    for (int b = lane; b < rmax; b += 32)
      V2s[(b * 8 + (r & 7)) * 4 + (r >> 3)] = (i2 < n && b < r2) ? V2[(long long)i2 * rmax + b] : 0.f;
  }
  // 16-byte chunk (8 ranks from a0) of the four points (i2b + warp + 8 q, i3)
  auto store_chunk = [&](int a0, const float (&lo4)[4][4], const float (&hi4)[4][4], bool zero) {
    if (i3 >= n) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i2 = i2b + warp + 8 * q;
      if (i2 >= n) continue;
      uint4 hi = make_uint4(0, 0, 0, 0), lo = make_uint4(0, 0, 0, 0);
      if (!zero) {
        float xs[8];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          xs[x] = lo4[q][x] * scale;
          xs[4 + x] = hi4[q][x] * scale;
        }
        split8_f16(xs, hi, lo);
      }
      const long long p = (long long)i2 * n + i3;
      unsigned char* tile = out + (unsigned long long)(p >> 7) * tile_bytes;
      const uint32_t off = kmajor_offset((int)(p & 127), a0 >> 3, kp >> 3);
      *(uint4*)(tile + off) = hi;
      *(uint4*)(tile + half_bytes + off) = lo;
    }
  };
  float lo4[4][4], hi4[4][4];
  // rank slices beyond r1: zero chunks, nothing to compute
  for (int a0 = (r1 + 7) & ~7; a0 < kp; a0 += 8) store_chunk(a0, lo4, hi4, true);
  // ranks in stages of four (a0 = 4h), two stages in flight: the asynchronous 4-byte copies of
  // stage h + 1 run while stage h is multiplied.  One copy instruction of a warp moves four
  // ranks of eight consecutive i3 (thread t: rank t % 4, column 8 k + t / 4), 128 contiguous
  // bytes of shared memory; zero fill outside the ranks / grid
  const int H = 2 * ((r1 + 7) >> 3);
  const int cx = lane & 3, cl = lane >> 2;
  auto issue = [&](int h) {
    float* buf = T1s + (size_t)(h & 1) * rmax * 128;
    const int a = 4 * h + cx;
    for (int e = warp; e < 4 * r2; e += 8) {
      const int b = e >> 2, col = 8 * (e & 3) + cl;
      const int i3c = t3 * AS_T3 + col;
      const bool in = a < r1 && i3c < n;
      const float* src = in ? T1 + ((long long)a * rmax + b) * n + i3c : T1;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(&buf[(b * 32 + col) * 4 + cx])),
                   "l"(src), "r"(in ? 4 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // stage h -> ac[i2 row q][rank x]
  auto stage = [&](int h, float (&ac)[4][4]) {
    if (h + 1 < H) {
      issue(h + 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int x = 0; x < 4; ++x) ac[q][x] = 0.f;
    const float4* T4 = reinterpret_cast<const float4*>(T1s + (size_t)(h & 1) * rmax * 128);
    const float4* V4 = reinterpret_cast<const float4*>(V2s);
    for (int b = 0; b < r2; ++b) {
      const float4 t = T4[b * 32 + lane], v = V4[b * 8 + warp];
      const float tv[4] = {t.x, t.y, t.z, t.w};
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int x = 0; x < 4; ++x) ac[q][x] = fmaf(vv[q], tv[x], ac[q][x]);
    }
    __syncthreads();                           // stage h's buffer is free for stage h + 2
  };
  if (H > 0) issue(0);
  for (int h = 0; h < H; h += 2) {
    stage(h, lo4);
    stage(h + 1, hi4);
    store_chunk(4 * h, lo4, hi4, false);
  }
}

// Interaction energy on the tensor-core path (Sec. 4.2, Eq. (4.7), Lemma 3.10): the Tucker
// value at a particle's grid point is sum_a V1[i1][a] T2[a][p], with T2[:, p] read from its tile
// (kp FP16 hi + lo values in 16-byte chunks, scaled by 2^(S-8)) instead of the r1 r2 terms of T1,
// which lie n apart in memory; the windows of the neighbours as on the CUDA-core path (FP64
// factors).  One warp per charged particle; one partial sum per CTA.
__global__ void __launch_bounds__(256)
energy_t2_kernel(DevView c, const float* __restrict__ V1, const unsigned char* __restrict__ T2t,
                 unsigned long long tile_bytes, int kp, const double* __restrict__ ewin, double* part) {
  __shared__ double red[8];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int mi = blockIdx.x * 8 + warp;
  double e = 0.0;
  if (mi < c.sc->n_nz) {
    const int p = c.nz_idx[mi];
    const int n = c.n, i1 = c.j[3 * p], i2 = c.j[3 * p + 1], i3 = c.j[3 * p + 2];
    const int r1 = c.sc->rank[0];
    const long long pt = (long long)i2 * n + i3;
    const unsigned char* tile = T2t + (unsigned long long)(pt >> 7) * tile_bytes;
    const int kc = kp >> 3;
    double v = 0.0;
    for (int ch = lane; ch < kc; ch += 32) {
      const uint32_t off = kmajor_offset((int)(pt & 127), ch, kc);
      const uint4 hi = *(const uint4*)(tile + off);
      const uint4 lo = *(const uint4*)(tile + tile_bytes / 2 + off);
      const __half2* h = reinterpret_cast<const __half2*>(&hi);
      const __half2* l = reinterpret_cast<const __half2*>(&lo);
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 fh = __half22float2(h[q]), fl = __half22float2(l[q]);
        const int a = 8 * ch + 2 * q;
        if (a < r1) s = fmaf(V1[(long long)i1 * c.rmax + a], fh.x + fl.x, s);
        if (a + 1 < r1) s = fmaf(V1[(long long)i1 * c.rmax + a + 1], fh.y + fl.y, s);
      }
      v += (double)s;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    v = ldexp(v, -(c.sc->t2_shift - 8)) + ewin[mi];   // plus the neighbours' windows
    const double z = c.Z[p];
    e = z * (v - z * c.sc->P_R0);
  }
  if (lane == 0) red[warp] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

int launch_energy_t2(Ctx& c, double* part, int blocks) {
  const unsigned long long tile_bytes = 4ull * AS_M * (unsigned long long)c.tc_kpad;   // hi + lo FP16
  energy_t2_kernel<<<blocks, 256, 0, c.stream>>>(make_view(c), (const float*)c.Z32, (const unsigned char*)c.T2,
                                                 tile_bytes, c.tc_kpad, c.ewin, part);
  return 1;
}

// The window part of every charged particle's value, sum_{nu in L(j)} z_nu U_nu(j): it needs
// only the particles and their bins, so it runs on the second stream beside the Gram and eigen
// stages.  One warp per charged particle.
__global__ void __launch_bounds__(256) energy_windows_kernel(DevView c, double* ewin) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int mi = blockIdx.x * 8 + warp;
  if (mi >= c.sc->n_nz) return;
  const int p = c.nz_idx[mi];
  double v = 0.0;
  window_add(c, c.j[3 * p], c.j[3 * p + 1], c.j[3 * p + 2], lane, v);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) ewin[mi] = v;
}

int launch_energy_windows(Ctx& c) {
  const int blocks = (c.maxN + 7) / 8 > 0 ? (c.maxN + 7) / 8 : 1;
  energy_windows_kernel<<<blocks, 256, 0, c.stream>>>(make_view(c), c.ewin);
  return 1;
}

// ------------------------------------------------------------------ assembly kernel
__global__ void __launch_bounds__(AS_THREADS, 1)
assemble_kernel(const AsmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_a_full[NA_MAX], bar_a_empty[NA_MAX];
  __shared__ __align__(8) uint64_t bar_list_full[2], bar_list_empty[2];
  __shared__ __align__(8) uint64_t bar_slot_full[NS_MAX], bar_slot_free[NS_MAX];
  __shared__ __align__(8) uint64_t bar_d_full[2], bar_d_empty[2], bar_drain;
  __shared__ __align__(8) uint64_t hdr_db[NS_MAX][2];     // B descriptors (hi, lo) of a pair
  __shared__ uint32_t hdr_id[NS_MAX][2];                   // instruction descriptor, column offset
  __shared__ int page_n[2], page_total[2], job_nw[NA_MAX];
  __shared__ int s_chunk, s_j0, s_stride, s_shiftT, s_shiftA, s_shiftB;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_s;
  volatile int* abort_flag = &abort_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  DevScalars* sc = g.sc;
  const int n = g.n;
  const long long np = (long long)n * n;
  const int r1 = sc->rank[0];
  const int gam = sc->gamma;

  if (tid == 0) {
    for (int s = 0; s < NA_MAX; ++s) {
      mbar_init(&bar_a_full[s], 1);
      mbar_init(&bar_a_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_list_full[b], 1);
      mbar_init(&bar_list_empty[b], NPW * NPG);
      mbar_init(&bar_d_full[b], 1);
      mbar_init(&bar_d_empty[b], NEPI);
    }
    for (int s = 0; s < NS_MAX; ++s) {
      mbar_init(&bar_slot_full[s], NPW);
      mbar_init(&bar_slot_free[s], 1);
    }
    mbar_init(&bar_drain, 1);
    abort_s = 0;
    // spread the CTAs over the i1 chunks in proportion to their work (same result in every CTA)
    double cost[32], tot = 0.0;
    for (int c = 0; c < g.nch; ++c) {
      cost[c] = g.cost_tile * g.ntiles + COST_WINDOW * (double)sc->chunk_w[c];
      tot += cost[c];
    }
    int cnt[32], used = 0;
    const int G = (int)gridDim.x;
    for (int c = 0; c < g.nch; ++c) {
      cnt[c] = 1 + (int)floor((double)(G - g.nch) * cost[c] / tot);
      used += cnt[c];
    }
    while (used < G) {
      int best = 0;
      for (int c = 1; c < g.nch; ++c)
        if (cost[c] * cnt[best] > cost[best] * cnt[c]) best = c;
      ++cnt[best];
      ++used;
    }
    int pre = 0, ch = g.nch - 1;
    for (int c = 0; c < g.nch; ++c) {
      if ((int)blockIdx.x < pre + cnt[c]) { ch = c; break; }
      pre += cnt[c];
    }
    s_chunk = ch;
    s_j0 = (int)blockIdx.x - pre;
    s_stride = cnt[ch];
    s_shiftT = operand_shift(sc, r1);
    // window operand scales: the table 2^sB p_k and A = 2^sA z p_k p_k stay below 2^14
    double fmax = 0.0;
    for (int k = 0; k < g.R_s; ++k) fmax = fmax > g.pk[(long long)(g.R_l + k) * g.L + (n - 1)] ? fmax : (double)g.pk[(long long)(g.R_l + k) * g.L + (n - 1)];
    const double zmax = (double)__uint_as_float(sc->zmax_bits);
    s_shiftB = (fmax > 0.0) ? 14 - exp2_above(fmax) : 0;
    s_shiftA = (fmax > 0.0 && zmax > 0.0) ? 14 - exp2_above(zmax * fmax * fmax) : 0;
    if (gam > g.gcap) atomicOr(&sc->flags, (unsigned)FLAG_WINDOWS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(g.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  const int chunk = s_chunk, j0 = s_j0, jstride = s_stride;
  const int c0 = chunk * g.Nc;
  const int cl = min(n, c0 + g.Nc) - 1;                 // last i1 row of this chunk
  const int njobs = (gam <= g.gcap && j0 < g.ntiles && c0 < n) ? (g.ntiles - 1 - j0) / jstride + 1 : 0;
  const int tw = 2 * g.gcap + 1;                        // rows d = -gcap .. gcap of the FP32 factors
  unsigned char* Bh = smem + g.off_bv;
  unsigned char* Bl = Bh + g.bv_half;
  unsigned char* Th = smem + g.off_tbl;
  unsigned char* Tl = Th + g.tbl_half;
  float* tab = (float*)(smem + g.off_tab);
  int4* lists = (int4*)(smem + g.off_list);

  // one-time staging by the whole CTA: the V1 rows of this chunk (B of the Tucker part, FP16
  // hi / lo, scaled by 2^8), the short-range factors p_k[d] (FP32, 8 ranks per row d, for the A
  // operands of the windows) and the factor table (B of the windows, FP16 hi / lo scaled by 2^sB, one 16-byte
  // row of 8 ranks per d = rho - D0)
  if (njobs > 0) {
    const int kc = g.kp >> 3;
    for (int e = tid; e < g.Nc * kc; e += AS_THREADS) {
      const int r = e / kc, k8 = e % kc, i1 = c0 + r;
      float x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int a = 8 * k8 + q;
        x[q] = (i1 < n && a < r1) ? 256.0f * g.V1[(long long)i1 * g.ldv + a] : 0.f;
      }
      uint4 hi, lo;
      split8_f16(x, hi, lo);
      const uint32_t off = kmajor_offset(r, k8, kc);
      *(uint4*)(Bh + off) = hi;
      *(uint4*)(Bl + off) = lo;
    }
    for (int e = tid; e < 8 * tw; e += AS_THREADS) {
      const int k = e & 7, d = (e >> 3) - g.gcap;
      tab[e] = (k < g.R_s && d >= -gam && d <= gam) ? g.pk[(long long)(g.R_l + k) * g.L + (n - 1) + d] : 0.f;
    }
    const float sBf = ldexpf(1.0f, s_shiftB);
    for (int rho = tid; rho < g.TR; rho += AS_THREADS) {
      const int d = rho - g.D0;
      float x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        x[k] = (k < g.R_s && d >= -gam && d <= gam) ? sBf * g.pk[(long long)(g.R_l + k) * g.L + (n - 1) + d] : 0.f;
      uint4 hi, lo;
      split8_f16(x, hi, lo);
      *(uint4*)(Th + (uint32_t)rho * 16u) = hi;
      *(uint4*)(Tl + (uint32_t)rho * 16u) = lo;
    }
    fence_proxy_async();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && njobs > 0) {
      const uint32_t sbo_t = (uint32_t)(g.kp >> 3) * 128u;    // T2 tiles and V1 (FP16)
      const uint64_t dBh = smem_desc(smem_addr(Bh), 128, sbo_t);
      const uint64_t dBl = smem_desc(smem_addr(Bl), 128, sbo_t);
      const uint64_t dA0 = smem_desc(smem_addr(smem + g.off_a), 128, sbo_t);
      const uint64_t dS0 = smem_desc(smem_addr(smem + g.off_slot), 128, 256);
      const uint64_t a_stage = (uint64_t)(2u * g.a_half) >> 4, a_lo = (uint64_t)g.a_half >> 4;
      const uint64_t s_step = (uint64_t)(2u * SLOT_HALF) >> 4, s_lo = (uint64_t)SLOT_HALF >> 4;
      const int ksteps = max(1, min(g.kp, (r1 + 15) & ~15) >> 4);
      const uint32_t id_main = idesc_f16(g.Nc);
      int st = 0, sl = 0;
      uint32_t stph = 0, slph = 0;
      bool ok = true;
      for (int t = 0; ok && t < njobs; ++t) {
        if (!wait_bar(&bar_a_full[st], stph, abort_flag, sc)) break;
        const int nw = job_nw[st];
        if (t >= 2 && !wait_bar(&bar_d_empty[t & 1], ((t - 2) >> 1) & 1, abort_flag, sc)) break;
        fence_after_sync();
        const uint32_t dT = tmem + (uint32_t)((t & 1) * g.dstride);
        const uint32_t dW = tmem + (uint32_t)((2 + (t & 1)) * g.dstride);
        const uint64_t ah = dA0 + (uint64_t)st * a_stage, al = ah + a_lo;
        for (int s = 0; s < ksteps; ++s) {
          const uint64_t ko = (uint64_t)s * 16u;           // 16 FP16 = 32 bytes per row
          mma_f16(dT, ah + ko, dBh + ko, id_main, s > 0 ? 1u : 0u);
          mma_f16(dT, ah + ko, dBl + ko, id_main, 1u);
          mma_f16(dT, al + ko, dBh + ko, id_main, 1u);
        }
        mma_commit(&bar_a_empty[st]);
        if (++st == g.na) { st = 0; stph ^= 1u; }
        const int npair = (nw + 1) >> 1;
        for (int q = 0; q < npair; ++q) {
          if (!wait_bar(&bar_slot_full[sl], slph, abort_flag, sc)) { ok = false; break; }
          fence_after_sync();
          const uint64_t bh = hdr_db[sl][0], bl = hdr_db[sl][1];
          const uint32_t idw = hdr_id[sl][0], dcol = hdr_id[sl][1];
          const uint64_t sh = dS0 + (uint64_t)sl * s_step, slo = sh + s_lo;
          mma_f16(dW + dcol, sh, bh, idw, q > 0 ? 1u : 0u);
          mma_f16(dW + dcol, sh, bl, idw, 1u);
          mma_f16(dW + dcol, slo, bh, idw, 1u);
          mma_commit(&bar_slot_free[sl]);
          if (++sl == g.ns) { sl = 0; slph ^= 1u; }
        }
        if (!ok) break;
        mma_commit(&bar_d_full[t & 1]);
      }
      // every MMA of this thread has completed before the tensor memory is released
      mma_commit(&bar_drain);
      drain_bar(&bar_drain, 0, sc);
    }
    __syncwarp();
  } else if (warp == WARP_SCHED) {
    // ------------------------------------------------------------ scheduler
    // Per job: the first page of its window list (the producers' input; it needs only a free
    // page), then the T2 tile (which waits for a free operand stage, that is for the MMAs of an
    // earlier job), then the rest of the list.  Copying the first page before the stage wait
    // keeps the producers from waiting behind the MMA issuer.
    int pg = 0, issued = 0, st = 0;
    uint32_t stph = 0;
    auto copy_page = [&](const int2 rg, int total, int off) -> bool {
      const int b = pg & 1;
      if (pg >= 2 && !warp_wait(&bar_list_empty[b], ((pg - 2) >> 1) & 1, abort_flag, sc)) return false;
      const int cnt = min(LIST_CAP, total - off);
      for (int i = lane; i < cnt; i += 32) lists[b * LIST_CAP + i] = g.rec[rg.x + off + i];
      if (lane == 0) { page_n[b] = cnt; page_total[b] = total; }
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_list_full[b]);
      ++pg;
      return true;
    };
    for (int t = 0; t < njobs; ++t) {
      const int T = j0 + t * jstride;
      int2 rg = make_int2(0, 0);
      if (g.rng) rg = g.rng[(long long)T * g.nch + chunk];
      const int total = rg.y - rg.x;
      if (!copy_page(rg, total, 0)) break;
      int ok = 1;
      if (lane == 0) {
        if (t >= g.na) ok = wait_bar(&bar_a_empty[st], stph ^ 1u, abort_flag, sc);
        if (ok) {
          job_nw[st] = total;
          mbar_expect_tx(&bar_a_full[st], (uint32_t)g.tile_bytes);
          bulk_load(smem + g.off_a + (size_t)st * 2 * g.a_half, g.T2t + (unsigned long long)T * g.tile_bytes,
                    (uint32_t)g.tile_bytes, &bar_a_full[st]);
          ++issued;
        }
      }
      if (++st == g.na) { st = 0; stph ^= 1u; }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      for (int off = LIST_CAP; off < total; off += LIST_CAP)
        if (!copy_page(rg, total, off)) { ok = 0; break; }
      if (!ok) break;
    }
    // the copies issued last have landed before the CTA exits
    if (lane == 0)
      for (int t = max(0, issued - g.na); t < issued; ++t)
        drain_bar(&bar_a_full[t % g.na], (uint32_t)(t / g.na) & 1u, sc);
    __syncwarp();
  } else if (warp < WARP_EPI) {
    // ------------------------------------------------------------ producers
    // Two groups of NPW warps.  Pair P (the running count of this CTA's window pairs over its
    // jobs) goes to slot P mod ns and is built by group P mod 2: thread pt of a group builds row
    // m = pt of both windows' A operands, every load issued before the arithmetic.  The
    // descriptors of a pair are written by lane 0 of one warp of its group.  Both groups walk
    // every page of a job's window list and release it.
    const int pw = warp - WARP_PROD;           // producer warp 0 .. NPG * NPW - 1
    const int gp = pw / NPW, wg = pw % NPW;    // group, warp within the group
    const int pt = (tid - WARP_PROD * 32) & (AS_M - 1);   // operand row m
    unsigned char* slot_base = smem + g.off_slot;
    const float sA = ldexpf(1.0f, s_shiftA);
    const uint32_t tbl_h = smem_addr(Th), tbl_l = smem_addr(Tl);
    const float4* tab4 = (const float4*)tab;
    int pg = 0;                                // list pages walked so far
    long long P0 = 0;                          // pairs of the earlier jobs
    // 16-column groups of the chunk that a pair reaches (all of them for the first pair of a
    // job, which overwrites the window accumulator), the table rows of its first row for each
    // window, and the descriptors
    auto header = [&](int slot, int q, int4 wa, int4 wb, bool has_b) {
      int s0, s1;
      if (q == 0) {
        s0 = 0;
        s1 = (g.Nc >> 4) - 1;
      } else {
        int lo1 = max(c0, wa.x - gam) - c0, hi1 = min(cl, wa.x + gam) - c0;
        if (has_b) {
          lo1 = min(lo1, max(c0, wb.x - gam) - c0);
          hi1 = max(hi1, min(cl, wb.x + gam) - c0);
        }
        s0 = lo1 >> 4;
        s1 = hi1 >> 4;
      }
      const int rho_a = c0 + 16 * s0 - wa.x + g.D0;
      const int rho_b = c0 + 16 * s0 - wb.x + g.D0;        // >= rho_a
      const uint32_t lbo = (uint32_t)(rho_b - rho_a) * 16u;
      hdr_db[slot][0] = smem_desc(tbl_h + (uint32_t)rho_a * 16u, lbo, 128);
      hdr_db[slot][1] = smem_desc(tbl_l + (uint32_t)rho_a * 16u, lbo, 128);
      hdr_id[slot][0] = idesc_f16(16 * (s1 - s0 + 1));
      hdr_id[slot][1] = (uint32_t)(16 * s0);
    };
    for (int t = 0; t < njobs; ++t) {
      const int T = j0 + t * jstride;
      int b = pg & 1;
      if (!warp_wait(&bar_list_full[b], (pg >> 1) & 1, abort_flag, sc)) break;
      const int nw = page_total[b];
      const int npair = (nw + 1) >> 1;
      const int npages = nw > 0 ? (nw + LIST_CAP - 1) / LIST_CAP : 1;
      int page = 0;                            // page of this job that pg refers to
      const long long p = (long long)T * AS_M + pt;
      const bool valid = p < np;
      const int i2 = valid ? (int)(p / n) : 0, i3 = valid ? (int)(p - (long long)i2 * n) : 0;
      bool ok = true;
      for (int q = gp; q < npair; q += NPG) {
        const int r0 = 2 * q;                  // first record of the pair (pages hold an even number)
        while (page < r0 / LIST_CAP) {         // on to the page of this pair
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar_list_empty[b]);
          ++pg;
          ++page;
          b = pg & 1;
          if (!warp_wait(&bar_list_full[b], (pg >> 1) & 1, abort_flag, sc)) { ok = false; break; }
        }
        if (!ok) break;
        const int pos = r0 - page * LIST_CAP, pn = page_n[b];
        int4 w[2];
        bool live[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          live[u] = pos + u < pn;
          // a missing second window repeats the first (zero operand, lbo 0)
          w[u] = lists[b * LIST_CAP + (live[u] ? pos + u : pos)];
        }
        if (live[1] && w[1].x > w[0].x) {      // chunk 0 of a pair: the window with the larger j1
          const int4 tmp = w[0];
          w[0] = w[1];
          w[1] = tmp;
        }
        // factor rows of the two windows, loaded before the slot wait
        float4 ra[2][2], rb[2][2];
        float zz[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int d2 = i2 - w[u].y, d3 = i3 - w[u].z;
          const bool in23 = live[u] && valid && d2 >= -gam && d2 <= gam && d3 >= -gam && d3 <= gam;
          const float4* r2 = tab4 + 2 * (in23 ? d2 + g.gcap : 0);
          const float4* r3 = tab4 + 2 * (in23 ? d3 + g.gcap : 0);
          ra[u][0] = r2[0];
          ra[u][1] = r2[1];
          rb[u][0] = r3[0];
          rb[u][1] = r3[1];
          zz[u] = in23 ? __int_as_float(w[u].w) * sA : 0.f;
        }
        const long long P = P0 + q;
        const int sl = (int)(P % g.ns);
        const uint32_t ph = (uint32_t)((P / g.ns) & 1);
        if (P >= g.ns && !warp_wait(&bar_slot_free[sl], ph ^ 1u, abort_flag, sc)) { ok = false; break; }
        unsigned char* sbh = slot_base + (size_t)sl * 2 * SLOT_HALF;
        unsigned char* sbl = sbh + SLOT_HALF;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const float z = zz[u];
          uint4 hi, lo;
          split_h2(z * ra[u][0].x * rb[u][0].x, z * ra[u][0].y * rb[u][0].y, hi.x, lo.x);
          split_h2(z * ra[u][0].z * rb[u][0].z, z * ra[u][0].w * rb[u][0].w, hi.y, lo.y);
          split_h2(z * ra[u][1].x * rb[u][1].x, z * ra[u][1].y * rb[u][1].y, hi.z, lo.z);
          split_h2(z * ra[u][1].z * rb[u][1].z, z * ra[u][1].w * rb[u][1].w, hi.w, lo.w);
          const uint32_t off = kmajor_offset(pt, u, 2);
          *(uint4*)(sbh + off) = hi;
          *(uint4*)(sbl + off) = lo;
        }
        if (lane == 0 && ((q / NPG) % NPW) == wg) header(sl, q, w[0], w[1], live[1]);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_slot_full[sl]);
      }
      if (!ok) break;
      // release this page and walk (and release) the job's remaining pages
      while (true) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_list_empty[b]);
        ++pg;
        ++page;
        if (page >= npages) break;
        b = pg & 1;
        if (!warp_wait(&bar_list_full[b], (pg >> 1) & 1, abort_flag, sc)) { ok = false; break; }
      }
      if (!ok) break;
      P0 += npair;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - WARP_EPI;
    const int q = warp & 3;                        // tensor-memory lanes 32q .. 32q+31
    const int half = ew >> 2;
    const int hw = g.Nc >> 1;
    const int cb = half * hw, ce = cb + hw;
    const float uT = ldexpf(1.0f, -s_shiftT), uW = ldexpf(1.0f, -(s_shiftA + s_shiftB));
    const int m = 32 * q + lane;
    float* stage = (float*)(smem + g.off_stage) + half * 32 * STG_ROW;
    for (int t = 0; t < njobs; ++t) {
      const int T = j0 + t * jstride;
      bool has_w = false;
      if (g.rng) { const int2 rg = g.rng[(long long)T * g.nch + chunk]; has_w = rg.y > rg.x; }
      if (!warp_wait(&bar_d_full[t & 1], (t >> 1) & 1, abort_flag, sc)) break;
      fence_after_sync();
      const long long p0 = (long long)T * AS_M;
      const int cnt = (int)min((long long)AS_M, np - p0);
      const uint32_t baseT = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((t & 1) * g.dstride);
      const uint32_t baseW = baseT + (uint32_t)(2 * g.dstride);
      for (int c = cb; c < ce; c += 32) {
        const int ncol = min(32, ce - c);
        uint32_t vt[32], vw[32];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (8 * u < ncol) tmem_ld8(baseT + (uint32_t)(c + 8 * u), vt + 8 * u);
        if (has_w) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (8 * u < ncol) tmem_ld8(baseW + (uint32_t)(c + 8 * u), vw + 8 * u);
        }
        tmem_wait_ld();
        if (g.staged) {
          // rows shifted to their 16-byte alignment in shared memory, then one bulk store of
          // the aligned middle of each plane row and scalar stores at its two ends; first, the
          // bulk stores of the previous group have read the staging rows
          if (lane < 8) bulk_wait_read();
          named_sync(1 + half, 128);
          const int o0 = (int)((((long long)(c0 + c)) * np + p0) & 3), ostep = (int)(np & 3);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < ncol) {
              float v = __uint_as_float(vt[j]) * uT;
              if (has_w) v = fmaf(__uint_as_float(vw[j]), uW, v);
              stage[j * STG_ROW + ((o0 + j * ostep) & 3) + m] = v;
            }
          }
          fence_proxy_async();
          named_sync(1 + half, 128);
          const int j = 8 * q + lane;                // staging row written out by this lane
          if (lane < 8 && j < ncol && c0 + c + j < n) {
            const long long a = (long long)(c0 + c + j) * np + p0;
            const int o = (int)(a & 3);
            const long long as = a + ((4 - o) & 3), ae = (a + cnt) & ~3ll;
            const float* row = stage + j * STG_ROW + o;
            for (long long x = a; x < min(as, a + cnt); ++x) g.P[x] = row[x - a];
            if (ae > as) bulk_store(g.P + as, row + (as - a), (uint32_t)((ae - as) * 4));
            for (long long x = max(ae, as); x < a + cnt; ++x) g.P[x] = row[x - a];
            bulk_commit();
          }
        } else if (m < cnt) {
          // lane m writes point p0 + m of the rows i1 = c0 + c + j: one 128-byte run per warp
          // and row (when the staging rows do not fit next to the operand rings)
          float* out = g.P + (long long)(c0 + c) * np + p0 + m;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < ncol && c0 + c + j < n) {
              float v = __uint_as_float(vt[j]) * uT;
              if (has_w) v = fmaf(__uint_as_float(vw[j]), uW, v);
              __stcs(out + (long long)j * np, v);
            }
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_d_empty[t & 1]);
    }
    if (g.staged && lane < 8) bulk_wait_all();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------------ window lists
// For every output tile (128 consecutive points p = i2 n + i3, all i1) the particles whose window
// (|i_l - j_l| <= gamma) reaches it, sorted by (j1, particle) so that the windows of one i1
// chunk are a contiguous range and the summation order does not depend on scheduling.  One CTA
// per tile scans the particles with nonzero charge (no global atomics).
__device__ __forceinline__ bool reaches_tile(int j2, int j3, long long p0, long long p1, int n, int g) {
  const int r0 = (int)(p0 / n), r1 = (int)(p1 / n);
  for (int r = r0; r <= r1; ++r) {
    const int lo3 = (r == r0) ? (int)(p0 - (long long)r * n) : 0;
    const int hi3 = (r == r1) ? (int)(p1 - (long long)r * n) : n - 1;
    if (j2 >= r - g && j2 <= r + g && j3 >= lo3 - g && j3 <= hi3 + g) return true;
  }
  return false;
}

__global__ void __launch_bounds__(256)
wl_count_kernel(const int* __restrict__ jidx, const int* __restrict__ nz_idx, const double* __restrict__ Z,
                DevScalars* sc, int n, int* count) {
  __shared__ int wsum[8];
  const int T = blockIdx.x, tid = threadIdx.x;
  const long long np = (long long)n * n;
  const long long p0 = (long long)T * AS_M, p1 = min(np, p0 + AS_M) - 1;
  const int g = sc->gamma, nnz = sc->n_nz;
  int cnt = 0;
  for (int m = tid; m < nnz; m += 256) {
    const int p = nz_idx[m];
    cnt += reaches_tile(jidx[3 * p + 1], jidx[3 * p + 2], p0, p1, n, g) ? 1 : 0;
    if (T == 0) atomicMax(&sc->zmax_bits, __float_as_uint(fabsf((float)Z[p])));
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((tid & 31) == 0) wsum[tid >> 5] = cnt;
  __syncthreads();
  if (tid == 0) {
    int s = 0;
    for (int w = 0; w < 8; ++w) s += wsum[w];
    count[T] = s;
  }
}

// one CTA per tile: collect its keys (j1 << 32 | particle), bitonic sort, write the records and
// the range of each i1 chunk
__global__ void __launch_bounds__(256)
wl_fill_kernel(const int* __restrict__ start, long long cap, const int* __restrict__ jidx,
               const int* __restrict__ nz_idx, const double* __restrict__ Z, DevScalars* sc, int n,
               int nch, int Nc, int4* rec, int2* rng) {
  __shared__ long long ks[WL_SORT_CAP];
  __shared__ int fill;
  const int T = blockIdx.x, tid = threadIdx.x;
  const long long np = (long long)n * n;
  const long long p0 = (long long)T * AS_M, p1 = min(np, p0 + AS_M) - 1;
  const int g = sc->gamma, nnz = sc->n_nz;
  const long long s = start[T], e = start[T + 1];
  const int len = (int)(e - s);
  if (len > WL_SORT_CAP || e > cap) {
    if (tid == 0) atomicOr(&sc->flags, (unsigned)FLAG_WINDOWS);
    for (int c = tid; c < nch; c += blockDim.x) rng[(long long)T * nch + c] = make_int2(0, 0);
    return;
  }
  if (tid == 0) fill = 0;
  __syncthreads();
  for (int m = tid; m < nnz; m += 256) {
    const int p = nz_idx[m];
    const int j1 = jidx[3 * p];
    if (reaches_tile(jidx[3 * p + 1], jidx[3 * p + 2], p0, p1, n, g)) {
      const int pos = atomicAdd(&fill, 1);       // order is restored by the sort below
      if (pos < len) ks[pos] = ((long long)j1 << 32) | (unsigned)p;
    }
  }
  int m2 = 1;
  while (m2 < len) m2 <<= 1;
  for (int i = len + tid; i < m2; i += blockDim.x) ks[i] = LLONG_MAX;
  __syncthreads();
  for (int k = 2; k <= m2; k <<= 1)
    for (int jx = k >> 1; jx > 0; jx >>= 1) {
      for (int i = tid; i < m2; i += blockDim.x) {
        const int ixj = i ^ jx;
        if (ixj > i) {
          const long long a = ks[i], b = ks[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { ks[i] = b; ks[ixj] = a; }
        }
      }
      __syncthreads();
    }
  for (int i = tid; i < len; i += blockDim.x) {
    const long long k = ks[i];
    const int p = (int)(unsigned)(k & 0xffffffffll);
    rec[s + i] = make_int4((int)(k >> 32), jidx[3 * p + 1], jidx[3 * p + 2], __float_as_int((float)Z[p]));
  }
  for (int c = tid; c < nch; c += blockDim.x) {
    const int lo_j = c * Nc - g, hi_j = min(n - 1, c * Nc + Nc - 1) + g;
    int lo = 0, hi = len;                       // first key with j1 >= lo_j
    while (lo < hi) { const int mid = (lo + hi) >> 1; if ((int)(ks[mid] >> 32) < lo_j) lo = mid + 1; else hi = mid; }
    int lo2b = lo, hi2b = len;                  // first key with j1 > hi_j
    while (lo2b < hi2b) { const int mid = (lo2b + hi2b) >> 1; if ((int)(ks[mid] >> 32) <= hi_j) lo2b = mid + 1; else hi2b = mid; }
    rng[(long long)T * nch + c] = make_int2((int)(s + lo), (int)(s + lo2b));
    if (lo2b > lo) atomicAdd(&sc->chunk_w[c], lo2b - lo);
  }
}

// scan of the counts (one CTA, chunked)
__global__ void wl_scan_kernel(const int* count, int nt, int* start) {
  __shared__ int scan[1024];
  const int Tn = blockDim.x, t = threadIdx.x;
  const int per = (nt + Tn - 1) / Tn;
  const int b0 = min(nt, t * per), b1 = min(nt, b0 + per);
  int s = 0;
  for (int b = b0; b < b1; ++b) s += count[b];
  scan[t] = s;
  __syncthreads();
  for (int o = 1; o < Tn; o <<= 1) {
    const int v = (t >= o) ? scan[t - o] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int pos = scan[t] - s;
  for (int b = b0; b < b1; ++b) { start[b] = pos; pos += count[b]; }
  if (t == Tn - 1) start[nt] = scan[t];
}

int launch_window_lists(Ctx& c) {
  if (c.R_s == 0) return 0;
  const int nT = c.tc_ntiles;
  wl_count_kernel<<<nT, 256, 0, c.stream>>>(c.j, c.nz_idx, c.Z, c.sc, c.n, c.wl_count);
  wl_scan_kernel<<<1, 1024, 0, c.stream>>>(c.wl_count, nT, c.wl_start);
  wl_fill_kernel<<<nT, 256, 0, c.stream>>>(c.wl_start, c.wl_cap, c.j, c.nz_idx, c.Z, c.sc, c.n,
                                           c.tc_nch, c.tc_Nc, c.wl_rec, c.wl_rng);
  return 3;
}

// ------------------------------------------------------------------ host planning
namespace {

// gamma of the device factor stage, evaluated on the host in FP64 with the same formulas
// (cell averages of the short-range Gaussians, Eq. (2.5); window criterion of Sec. 2.3)
int host_gamma(const Ctx& c) {
  const int n = c.n, R = c.R, R_l = c.R_l;
  const double h = c.h, hq = c.cfg.h_q, u0 = c.cfg.u0;
  auto p = [&](int k, int d) {
    const double t = std::exp(u0 + k * hq);
    const double a = 1.1283791670955126 * hq * t;
    const double x = std::fabs((double)d) * h;
    const double lo = t * (x - 0.5 * h), hi = t * (x + 0.5 * h);
    const double diff = (lo > 0.5) ? (std::erfc(lo) - std::erfc(hi)) : (std::erf(hi) - std::erf(lo));
    return std::cbrt(a) * (0.88622692545275801 / (t * h)) * diff;
  };
  double PR0 = 0.0;
  for (int k = 0; k < R; ++k) { const double v = p(k, 0); PR0 += v * v * v; }
  const double delta = c.cfg.delta_rel * PR0;
  int cnt = 0;
  for (int gg = 0; gg <= n - 2; ++gg) {
    double v = 0.0;
    for (int k = R_l; k < R; ++k) { const double p0 = p(k, 0); v += p(k, gg + 1) * p0 * p0; }
    if (v > delta) ++cnt;
  }
  return cnt < n - 1 ? cnt : n - 1;
}

inline size_t al128(size_t x) { return (x + 127) & ~(size_t)127; }

struct Layout {
  size_t bv_half, a_half, tbl_half, tab, list, stage;
  int TR, D0;
};

Layout layout_of(const Ctx& c) {
  Layout L;
  L.bv_half = al128((size_t)c.tc_Nc * c.tc_kpad * 2);
  L.a_half = (size_t)AS_M * c.tc_kpad * 2;
  L.D0 = c.tc_Nc + c.gamma_cap;
  L.TR = L.D0 + c.tc_Nc + c.gamma_cap + 16;
  L.tbl_half = al128((size_t)L.TR * 16);
  L.tab = al128((size_t)8 * (2 * c.gamma_cap + 1) * 4);
  L.list = (size_t)2 * LIST_CAP * 16;
  L.stage = (size_t)2 * 32 * STG_ROW * 4;
  return L;
}

size_t smem_total(const Layout& L, int na, int ns, bool staged) {
  return 2 * L.bv_half + (size_t)na * 2 * L.a_half + (size_t)ns * 2 * SLOT_HALF + 2 * L.tbl_half + L.tab +
         L.list + (staged ? L.stage : 0);
}

}  // namespace

bool plan_assemble(Ctx& c) {
  if (c.fp64) return false;
  const char* env = std::getenv("RS_RECON_PATH");
  if (env && std::strcmp(env, "cuda") == 0) return false;
  if (c.R_s > 8) return false;                            // one 8-wide K chunk per window
  const int n = c.n;
  const int gh = host_gamma(c);
  c.gamma_cap = gh + 1 < n - 1 ? gh + 1 : n - 1;
  c.tc_kpad = (c.rmax + 15) & ~15;
  c.tc_nch = (n + 127) / 128;
  const int per = (n + c.tc_nch - 1) / c.tc_nch;
  c.tc_Nc = (per + 15) & ~15;
  c.tc_ntiles = (int)(((long long)n * n + AS_M - 1) / AS_M);
  if (c.tc_nch > 32) return false;
  const Layout L = layout_of(c);
  const size_t limit = (size_t)(SMEM_LIMIT - SMEM_RESERVE);
  // deepest operand rings that fit, with the staged epilogue (faster stores: the protein
  // workload's assembly 431 -> 416 us at a split refitted to it, with six window slots instead of
  // eight) unless dropping its staging rows buys a ring more than one step deeper (large ranks)
  // (at least two window slots: the two producer groups build alternate pairs)
  const int choices[5][2] = {{2, 8}, {2, 6}, {2, 4}, {1, 4}, {1, 2}};
  int best[2] = {-1, -1};
  for (int staged = 1; staged >= 0; --staged)
    for (int i = 0; i < 5; ++i)
      if (smem_total(L, choices[i][0], choices[i][1], staged != 0) <= limit) {
        best[staged] = i;
        break;
      }
  if (best[0] < 0) return false;
  c.tc_staged = best[1] >= 0 && best[1] <= best[0] + 1;   // staging may cost one ring step
  const int pick = c.tc_staged ? best[1] : best[0];
  c.tc_na = choices[pick][0];
  c.tc_ns = choices[pick][1];
  c.tc_smem = smem_total(L, c.tc_na, c.tc_ns, c.tc_staged);
  // the T2 tile kernel stages 8 rank slices of T1 for 32 i3 plus 32 rows of V2
  if ((size_t)1152 * c.rmax > limit) return false;
  // window list entries: every particle reaches at most the tiles of 2 gamma + 1 rows of
  // n points plus one tile
  const long long per_particle = ((long long)(2 * c.gamma_cap + 1) * n + AS_M - 1) / AS_M + 2;
  long long cap = (long long)c.maxN * std::min<long long>(c.tc_ntiles, per_particle);
  if (cap < 1) cap = 1;
  if (cap > INT_MAX / 2) return false;
  c.wl_cap = cap;
  return true;
}

size_t t2_tile_bytes(const Ctx& c) {
  return (size_t)c.tc_ntiles * 2 * layout_of(c).a_half;
}

int launch_t2_tiles(Ctx& c) {
  const size_t shm = (size_t)1152 * c.rmax;
  const dim3 grid((c.n + AS_T3 - 1) / AS_T3, (c.n + TT_ROWS - 1) / TT_ROWS);
  t2_tiles_kernel<<<grid, 256, shm, c.stream>>>((const float*)c.T1, c.Z32 + (size_t)c.n * c.rmax, c.n,
                                                c.rmax, c.tc_kpad, c.tc_ntiles, c.sc,
                                                (unsigned char*)c.T2, 2 * layout_of(c).a_half);
  return 1;
}

int launch_assemble(Ctx& c, float* out) {
  const Layout L = layout_of(c);
  AsmArgs g;
  g.T2t = (const unsigned char*)c.T2;
  g.tile_bytes = 2 * L.a_half;
  g.V1 = c.Z32;
  g.ldv = c.rmax;
  g.pk = c.pk32;
  g.rec = c.wl_rec;
  g.rng = c.R_s > 0 ? c.wl_rng : nullptr;
  g.P = out;
  g.sc = c.sc;
  g.n = c.n;
  g.L = c.L;
  g.R_l = c.R_l;
  g.R_s = c.R_s;
  g.nch = c.tc_nch;
  g.Nc = c.tc_Nc;
  g.kp = c.tc_kpad;
  g.gcap = c.gamma_cap;
  g.TR = L.TR;
  g.D0 = L.D0;
  g.ntiles = c.tc_ntiles;
  int ds = 16;
  while (ds < c.tc_Nc) ds <<= 1;
  g.dstride = ds;
  g.tmem_cols = 4 * ds < 32 ? 32 : 4 * ds;
  g.na = c.tc_na;
  g.ns = c.tc_ns;
  g.off_bv = 0;
  g.off_a = (uint32_t)(2 * L.bv_half);
  g.off_slot = (uint32_t)(g.off_a + (size_t)c.tc_na * 2 * L.a_half);
  g.off_tbl = (uint32_t)(g.off_slot + (size_t)c.tc_ns * 2 * SLOT_HALF);
  g.off_tab = (uint32_t)(g.off_tbl + 2 * L.tbl_half);
  g.off_list = (uint32_t)(g.off_tab + L.tab);
  g.off_stage = (uint32_t)(g.off_list + L.list);
  g.staged = c.tc_staged ? 1 : 0;
  g.cost_tile = c.tc_staged ? COST_TILE_STAGED : COST_TILE;
  g.bv_half = (uint32_t)L.bv_half;
  g.a_half = (uint32_t)L.a_half;
  g.tbl_half = (uint32_t)L.tbl_half;
  if (c.tc_grid == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c.tc_grid = sms > c.tc_nch ? sms : c.tc_nch;
  }
  assemble_kernel<<<c.tc_grid, AS_THREADS, c.tc_smem, c.stream>>>(g);
  return 1;
}

cudaError_t set_attributes_tc(int optin) {
  cudaError_t e = allow_max_dynamic_smem((const void*)t2_tiles_kernel, optin);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)assemble_kernel, optin);
  return e;
}

}  // namespace rs
