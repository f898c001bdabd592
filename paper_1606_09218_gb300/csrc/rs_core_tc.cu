// Tensor-core (tcgen05) contraction of the Tucker core on the FP32 bulk path:
//
//   beta[a][b][c] = sum_K z_K q1[K][a] q2[K][b] q3[K][c]        (Eq. (6.2): beta = xi x_1 U~1
//                                                                 x_2 U~2 x_3 U~3, w^3 = |z|)
//
// with K = (charged particle p, long-range index k) and q_l[K] = Qp_l[j_l(p)][k], the
// projection of the shifted factor onto the Tucker basis of mode l.  As a GEMM over K:
// A[a][K] = z_K q1[K][a] (M = 128 rows a) and B[(b,c)][K] = q2[K][b] q3[K][c] (N = 64 pairs,
// 8 b x 8 c), both built on the fly from the L2-resident projections and split into FP16
// hi + lo (three products hi*hi + hi*lo + lo*hi, 2^-22 relative), accumulated in FP32 in
// tensor memory over segments of 64 terms (one chunk, twelve MMAs).  Every segment is folded
// into an FP32 (hi, lo) pair per output with an error-free two-sum, and a work unit (an output
// tile and a slice of K) adds its pairs to beta in FP64.  The tensor cores' FP32 accumulation
// is coarser than round-to-nearest: measured on the protein workload (n = 513, eps = 1e-6)
// against the CUDA-core contraction with two-sum chunks, the potentials differ by 4e-7 with
// 64-term segments, 9e-7 with 256 and 2e-6 with 1024 (energies by 2e-6 .. 3e-5 relative), so
// segments stay at 64 terms.
//
// Two forms.  core_tc_kernel (this header) builds both operands per output tile; the
// Khatri-Rao form further down (core_w_kernel + core_kr_kernel) forms z q1 q2 once per solve
// and streams it, and is the default on the FP32 path wherever its operand window covers K in
// at most KR_MAX_PASSES passes (every workload here); core_tc_kernel remains for larger
// problems at tolerances of at least 1e-5, the CUDA-core contraction below that.
//
// Operand scales: A carries 2^sA with 2^sA max|z| max|q| < 2^14 and B 2^sB with
// 2^sB max|q|^2 < 2^14 (exact powers of two, removed when the units add to beta).
//
// CTA (one per SM, 16 warps):
//   warp 0      tensor-memory owner; lane 0 issues the MMAs into two accumulator buffers
//   warps 1-7   producers: A and B chunks of 64 K terms -> ring of four stages
//   warps 8-15  epilogue: a segment's accumulator -> (hi, lo) registers; FP64 atomics per unit
// Every wait is bounded (FLAG_TIMEOUT, abort flag, tensor memory released before return).
#include <algorithm>

#include "rs_internal.cuh"
#include "rs_tcgen05.cuh"

namespace rs {
namespace {

constexpr int CT_M = 128;                    // a rows of a tile (tensor-memory lanes)
constexpr int CT_N = 64;                     // (b, c) pairs of a tile: 8 b x 8 c
constexpr int CT_KC = 64;                    // K terms of one chunk (four K = 16 MMA steps)
constexpr int CT_SEG = 1;                    // chunks of one accumulation segment (64 terms)
constexpr int CT_STAGES = 4;
constexpr int CT_PROD = 7;                   // producer warps (16 warps: 128 registers a thread)
constexpr int CT_EPI = 8;                    // epilogue warps
constexpr int CT_THREADS = 32 * (1 + CT_PROD + CT_EPI);
constexpr uint32_t CT_A_HALF = CT_M * CT_KC * 2;                  // FP16 hi or lo, bytes
constexpr uint32_t CT_B_HALF = CT_N * CT_KC * 2;
constexpr uint32_t CT_STAGE = 2 * CT_A_HALF + 2 * CT_B_HALF;      // 48 KB
constexpr uint32_t CT_SMEM = CT_STAGES * CT_STAGE;                // 192 KB
constexpr uint32_t CT_TMEM_COLS = 2 * CT_N;

struct CoreArgs {
  const float* Qp;        // [3][n][R_l][rmax]
  const int4* meta;       // per K: row offsets of q1, q2, q3 in Qp, z (float bits)
  DevScalars* sc;
  double* beta64;         // [rmax][rmax][rmax], zeroed by the caller
  int rmax, R_l;
};

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// unit u -> output tile (a0, b0, c0) and chunk range [cb, ce) of K
struct Unit {
  int a0, b0, c0;
  long long cb, ce;
};

struct UnitPlan {
  int Mt, nc8, Nt, S;
  long long Kc, units;
  __device__ Unit unit(long long u) const {
    Unit t;
    const int s = (int)(u % S);
    const long long rest = u / S;
    const int nt = (int)(rest % Nt), m = (int)(rest / Nt);
    t.a0 = m * CT_M;
    t.b0 = (nt / nc8) * 8;
    t.c0 = (nt % nc8) * 8;
    t.cb = Kc * s / S;
    t.ce = Kc * (s + 1) / S;
    return t;
  }
};

__device__ __forceinline__ UnitPlan plan_units(const DevScalars* sc, int R_l, int grid) {
  UnitPlan P;
  const int r1 = sc->rank[0], r2 = sc->rank[1], r3 = sc->rank[2];
  const long long Ktot = (long long)sc->n_nz * R_l;
  P.Mt = (r1 + CT_M - 1) / CT_M;
  P.nc8 = (r3 + 7) / 8;
  P.Nt = ((r2 + 7) / 8) * P.nc8;
  P.Kc = (Ktot + CT_KC - 1) / CT_KC;
  const long long nseg = (P.Kc + CT_SEG - 1) / CT_SEG;
  const long long tiles = (long long)P.Mt * P.Nt;
  long long S = tiles > 0 ? (2ll * grid + tiles - 1) / tiles : 1;
  if (S > nseg) S = nseg;
  if (S < 1) S = 1;
  P.S = (int)S;
  P.units = (tiles > 0 && P.Kc > 0) ? tiles * S : 0;
  return P;
}

}  // namespace

// per K = (charged particle, long k): the Qp row offsets of its three projected factors and its
// charge; the largest |z| for the operand scale
__global__ void __launch_bounds__(256)
core_meta_kernel(const int* __restrict__ jidx, const int* __restrict__ nz_idx, const double* __restrict__ Z,
                 int n, int rmax, int R_l, DevScalars* sc, int4* meta) {
  const long long K = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long Ktot = (long long)sc->n_nz * R_l;
  float zm = 0.f;
  if (K < Ktot) {
    const int p = nz_idx[K / R_l], k = (int)(K % R_l);
    const long long sL = (long long)n * R_l * rmax;
    const float z = (float)Z[p];
    meta[K] = make_int4((int)(((long long)jidx[3 * p] * R_l + k) * rmax),
                        (int)(sL + ((long long)jidx[3 * p + 1] * R_l + k) * rmax),
                        (int)(2 * sL + ((long long)jidx[3 * p + 2] * R_l + k) * rmax), __float_as_int(z));
    zm = fabsf(z);
  }
  for (int o = 16; o > 0; o >>= 1) zm = fmaxf(zm, __shfl_xor_sync(0xffffffffu, zm, o));
  if ((threadIdx.x & 31) == 0 && zm > 0.f) atomicMax(&sc->zmax_bits, __float_as_uint(zm));
}

__global__ void __launch_bounds__(CT_THREADS, 1) core_tc_kernel(CoreArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full[CT_STAGES], bar_empty[CT_STAGES];
  __shared__ __align__(8) uint64_t bar_dfull[2], bar_dempty[2], bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_s;
  volatile int* abort_flag = &abort_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  DevScalars* sc = g.sc;
  const int r1 = sc->rank[0], r2 = sc->rank[1], r3 = sc->rank[2];
  const long long Ktot = (long long)sc->n_nz * g.R_l;
  const UnitPlan P = plan_units(sc, g.R_l, (int)gridDim.x);
  const float qmax = __uint_as_float(sc->qmax_bits), zmax = __uint_as_float(sc->zmax_bits);
  const int sA = (qmax > 0.f && zmax > 0.f) ? max(-100, min(100, 14 - exp2_above((double)zmax * qmax))) : 0;
  const int sB = (qmax > 0.f) ? max(-100, min(100, 14 - exp2_above((double)qmax * qmax))) : 0;
  const double pfx = ldexp(1.0, beta_fx_shift(sc, g.R_l));   // fixed-point scale of the beta sums

  if (tid == 0) {
    for (int s = 0; s < CT_STAGES; ++s) {
      mbar_init(&bar_full[s], CT_PROD);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_dfull[b], 1);
      mbar_init(&bar_dempty[b], CT_EPI);
    }
    mbar_init(&bar_drain, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(CT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && P.units > 0) {
      const uint64_t dA = smem_desc(smem_addr(smem), 128, (CT_KC / 8) * 128);
      const uint64_t dB = smem_desc(smem_addr(smem + 2 * CT_A_HALF), 128, (CT_KC / 8) * 128);
      const uint64_t st_step = (uint64_t)CT_STAGE >> 4;
      const uint64_t a_lo = (uint64_t)CT_A_HALF >> 4, b_lo = (uint64_t)CT_B_HALF >> 4;
      const uint32_t idesc = idesc_f16(CT_N, CT_M);
      long long gc = 0, gseg = 0;
      bool ok = true;
      for (long long u = blockIdx.x; ok && u < P.units; u += gridDim.x) {
        const Unit t = P.unit(u);
        for (long long c = t.cb; c < t.ce; ++c) {
          const long long cl = c - t.cb;
          const bool seg_start = (cl % CT_SEG) == 0;
          const int buf = (int)(gseg & 1);
          if (seg_start && gseg >= 2 && !wait_bar(&bar_dempty[buf], (uint32_t)((gseg - 2) >> 1) & 1u, abort_flag, sc)) {
            ok = false;
            break;
          }
          const int st = (int)(gc % CT_STAGES);
          if (!wait_bar(&bar_full[st], (uint32_t)(gc / CT_STAGES) & 1u, abort_flag, sc)) {
            ok = false;
            break;
          }
          fence_after_sync();
          const uint32_t d = tmem + (uint32_t)(buf * CT_N);
          const uint64_t ah = dA + (uint64_t)st * st_step, al = ah + a_lo;
          const uint64_t bh = dB + (uint64_t)st * st_step, bl = bh + b_lo;
#pragma unroll
          for (int s4 = 0; s4 < CT_KC / 16; ++s4) {
            const uint64_t ko = (uint64_t)s4 * 16u;        // 16 FP16 = 32 bytes per row = 2 chunks
            mma_f16(d, ah + ko, bh + ko, idesc, (seg_start && s4 == 0) ? 0u : 1u);
            mma_f16(d, ah + ko, bl + ko, idesc, 1u);
            mma_f16(d, al + ko, bh + ko, idesc, 1u);
          }
          mma_commit(&bar_empty[st]);
          ++gc;
          if ((cl % CT_SEG) == CT_SEG - 1 || c == t.ce - 1) {
            mma_commit(&bar_dfull[buf]);
            ++gseg;
          }
        }
      }
      // every MMA of this thread has completed before the tensor memory is released
      mma_commit(&bar_drain);
      drain_bar(&bar_drain, 0, sc);
    }
    __syncwarp();
  } else if (warp <= CT_PROD) {
    // ------------------------------------------------------------ producers
    const int pt = tid - 32;                          // 0 .. 255
    const float fA = ldexpf(1.0f, sA), fB = ldexpf(1.0f, sB);
    long long gc = 0;
    bool ok = true;
    for (long long u = blockIdx.x; ok && u < P.units; u += gridDim.x) {
      const Unit t = P.unit(u);
      const long long kend = min(Ktot, t.ce * CT_KC);
      for (long long c = t.cb; c < t.ce; ++c) {
        const int st = (int)(gc % CT_STAGES);
        if (gc >= CT_STAGES && !warp_wait(&bar_empty[st], (uint32_t)(gc / CT_STAGES - 1) & 1u, abort_flag, sc)) {
          ok = false;
          break;
        }
        unsigned char* base = smem + (size_t)st * CT_STAGE;
        const long long K0 = c * CT_KC;
        // tasks: 128 rows x 8 K groups of A, then 64 rows x 8 K groups of B
        //   A[a][K] = 2^sA z_K q1[K][a]
        //   B[(b,c)][K] = 2^sB q2[K][b] q3[K][c], row = 8 (b - b0) + (c - c0)
        for (int task = pt; task < CT_M * 8 + CT_N * 8; task += 32 * CT_PROD) {
          float x[8];
          uint32_t off, hoff;
          if (task < CT_M * 8) {                      // warp-uniform (1024 is a multiple of 32)
            const int row = task & (CT_M - 1), kg = task >> 7, a = t.a0 + row;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const long long K = K0 + 8 * kg + q;
              x[q] = 0.f;
              if (K < kend && a < r1) {
                const int4 mt = g.meta[K];
                x[q] = fA * __int_as_float(mt.w) * g.Qp[mt.x + a];
              }
            }
            off = kmajor_offset(row, kg, CT_KC / 8);
            hoff = CT_A_HALF;
          } else {
            const int t2 = task - CT_M * 8;
            const int row = t2 & (CT_N - 1), kg = t2 >> 6;
            const int b = t.b0 + (row >> 3), cc = t.c0 + (row & 7);
            const bool live = b < r2 && cc < r3;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const long long K = K0 + 8 * kg + q;
              x[q] = 0.f;
              if (K < kend && live) {
                const int4 mt = g.meta[K];
                x[q] = fB * g.Qp[mt.y + b] * g.Qp[mt.z + cc];
              }
            }
            off = 2 * CT_A_HALF + kmajor_offset(row, kg, CT_KC / 8);
            hoff = CT_B_HALF;
          }
          uint4 hi, lo;
          split8_f16(x, hi, lo);
          *(uint4*)(base + off) = hi;
          *(uint4*)(base + off + hoff) = lo;
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_full[st]);
        ++gc;
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 1 - CT_PROD;               // 0 .. 7
    const int q = warp & 3;                          // tensor-memory lanes 32q .. 32q + 31
    const int half = ew >> 2;                        // columns 32 half .. 32 half + 31
    const double unscale = ldexp(1.0, -(sA + sB));
    long long gseg = 0;
    bool ok = true;
    for (long long u = blockIdx.x; ok && u < P.units; u += gridDim.x) {
      const Unit t = P.unit(u);
      const long long nseg = (t.ce - t.cb + CT_SEG - 1) / CT_SEG;
      float hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        hi[j] = 0.f;
        lo[j] = 0.f;
      }
      for (long long sg = 0; sg < nseg; ++sg) {
        const int buf = (int)(gseg & 1);
        if (!warp_wait(&bar_dfull[buf], (uint32_t)(gseg >> 1) & 1u, abort_flag, sc)) {
          ok = false;
          break;
        }
        fence_after_sync();
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * CT_N + 32 * half);
#pragma unroll
        for (int u8 = 0; u8 < 4; ++u8) {
          uint32_t v[8];
          tmem_ld8(ta + (uint32_t)(8 * u8), v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) two_sum_acc(hi[8 * u8 + j], lo[8 * u8 + j], __uint_as_float(v[j]));
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_dempty[buf]);
        ++gseg;
      }
      if (!ok) break;
      const int a = t.a0 + 32 * q + lane;
      if (a < r1) {
        // columns 32 half + j: b = b0 + 4 half + j / 8, c = c0 + j % 8
        unsigned long long* out = reinterpret_cast<unsigned long long*>(g.beta64) +
                                  ((long long)a * g.rmax + t.b0 + 4 * half) * g.rmax + t.c0;
        const int nb = min(4, r2 - t.b0 - 4 * half), nc = min(8, r3 - t.c0);
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if ((j >> 3) < nb && (j & 7) < nc)
            atomicAdd(out + (j >> 3) * g.rmax + (j & 7), beta_fx(((double)hi[j] + (double)lo[j]) * unscale, pfx));
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CT_TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------------ Khatri-Rao form
// The same contraction with the Khatri-Rao product of the first two modes formed once:
//   W[(a, b)][K] = z_K q1[K][a] q2[K][b]     (rows rho = a r2 + b, r1 r2 of them)
//   beta[a][b][c] = sum_K W[(a, b)][K] q3[K][c]
// a GEMM with M = 128 pairs (a, b), N = cn values of c (64 when r3 <= 64, else 96, so that one
// tile holds every c up to r3 = 96 and each W block is read once) and K in chunks of 64 terms.
// core_w_kernel writes W and q3 as FP16 hi / lo chunks in the canonical K-major layout of the
// MMA operands (32 KB per 128 pairs and chunk, cn x 256 bytes per cn values of c and chunk),
// scaled by 2^sA and 2^sB as above.  core_kr_kernel copies them into a ring of shared-memory stages with bulk copies (one
// loader warp), accumulates 64-term segments in tensor memory, folds every segment into FP32
// (hi, lo) pairs and adds each unit's pairs to beta as fixed-point integers.  Against the producers
// of core_tc_kernel every operand value is built once instead of once per output tile, and all
// 128 rows of a tile are live (r1 r2 pairs instead of r1 < 128 rows a).
//
// The operands of all K would take Mt Kc (32 KB + q3 blocks) at the largest ranks (Mt tiles of
// pairs, Kc chunks); a workspace of a fixed size holds a window of chunks, and the K range is covered in
// `passes` windows (the same number for every launch, fixed on the host from the rank cap and the
// particle capacity; each window holds ceil(Kc / passes) chunks of the actual ranks).

constexpr uint32_t KR_A = 2 * CT_A_HALF;          // one A block: hi and lo of 128 pairs x 64 K
// one B block: hi and lo of cn values of c x 64 K (cn = 64 when r3 <= 64, else 96)
__host__ __device__ constexpr uint32_t kr_b(int cn) { return 2u * (uint32_t)cn * CT_KC * 2u; }
constexpr uint32_t KR_SMEM = CT_SMEM;             // stage ring: 4 stages at cn = 64, 3 at cn = 96
constexpr uint32_t KR_TMEM_COLS = 256;            // two accumulators of up to 96 columns
constexpr int KR_EPI = 8;
constexpr int KR_THREADS = 32 * (2 + KR_EPI);     // MMA warp, loader warp, 8 epilogue warps
constexpr int KR_MAX_PASSES = 8;

struct KrGeom {
  int mt, nt, cn, w;       // tiles of 128 pairs, tiles of cn values of c, chunks of a window
  long long kc, ktot;      // chunks and terms of K
};

__device__ __forceinline__ KrGeom kr_geom(const DevScalars* sc, int R_l, int passes) {
  KrGeom G;
  G.ktot = (long long)sc->n_nz * R_l;
  G.kc = (G.ktot + CT_KC - 1) / CT_KC;
  G.mt = (sc->rank[0] * sc->rank[1] + CT_M - 1) / CT_M;
  G.cn = sc->rank[2] <= 64 ? 64 : 96;               // one c tile up to r3 = 96: each A block read once
  G.nt = (sc->rank[2] + G.cn - 1) / G.cn;
  G.w = (int)((G.kc + passes - 1) / passes);
  return G;
}

// A = 2^sA z q1 q2 with 2^sA max|z| max|q|^2 < 2^14, B = 2^sB q3 with 2^sB max|q| < 2^14
__device__ __forceinline__ void kr_scales(const DevScalars* sc, int& sA, int& sB) {
  const float qmax = __uint_as_float(sc->qmax_bits), zmax = __uint_as_float(sc->zmax_bits);
  sA = (qmax > 0.f && zmax > 0.f) ? max(-100, min(100, 14 - exp2_above((double)zmax * qmax * qmax))) : 0;
  sB = (qmax > 0.f) ? max(-100, min(100, 14 - exp2_above((double)qmax))) : 0;
}

// Operands of window `pass`: blocks (tile, chunk - first chunk of the window), wstride chunks per
// tile in the workspace.  A task is a chunk and KR_AB values of a (all b), or a chunk's q3 tiles;
// one 256-thread block per task, grid-stride.  Warp g builds K group g (8 terms) of the rows
// (a, b), lane = b - b0: it keeps q2[K][b] of its 8 terms in registers and reads 2^sA z q1[K][a]
// from shared memory (one broadcast per 8 terms), so a value of W costs one multiply and its
// FP16 split.  The rows past the last pair of the last tile are written as zeros.
constexpr int KR_AB = 8;

__global__ void __launch_bounds__(256, 4)
core_w_kernel(const float* __restrict__ Qp, const int4* __restrict__ meta, const DevScalars* sc, int R_l,
              int passes, int pass, int wstride, unsigned char* __restrict__ W, unsigned char* __restrict__ B3) {
  __shared__ int4 sm[CT_KC];
  __shared__ __align__(16) float zq1[KR_AB][CT_KC];
  const int r1 = sc->rank[0], r2 = sc->rank[1], r3 = sc->rank[2];
  const KrGeom G = kr_geom(sc, R_l, passes);
  const long long c0 = (long long)pass * G.w;
  const int wl = (int)max(0ll, min((long long)G.w, G.kc - c0));    // chunks of this window
  const int nab = (r1 + KR_AB - 1) / KR_AB;
  const long long ntask = (long long)(nab + 1) * wl;
  if (ntask == 0 || G.mt == 0) return;
  int sA, sB;
  kr_scales(sc, sA, sB);
  const float fA = ldexpf(1.0f, sA), fB = ldexpf(1.0f, sB);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, pairs = r1 * r2;
  for (long long t = blockIdx.x; t < ntask; t += gridDim.x) {
    const int ab = (int)(t / wl), cl = (int)(t % wl);
    const long long K0 = (c0 + cl) * CT_KC;
    __syncthreads();                                   // the previous task's reads of sm, zq1
    if (tid < CT_KC) sm[tid] = K0 + tid < G.ktot ? meta[K0 + tid] : make_int4(0, 0, 0, 0);
    __syncthreads();
    if (ab < nab) {
      const int a0 = ab * KR_AB, na = min(KR_AB, r1 - a0);
      for (int e = tid; e < KR_AB * CT_KC; e += 256) {
        const int i = e >> 6, kk = e & (CT_KC - 1);
        const int4 mt = sm[kk];
        zq1[i][kk] = (i < na && K0 + kk < G.ktot) ? fA * __int_as_float(mt.w) * Qp[mt.x + a0 + i] : 0.f;
      }
      __syncthreads();
      for (int b0 = 0; b0 < r2; b0 += 32) {
        const int b = b0 + lane;
        if (b >= r2) continue;
        float q2v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int kk = 8 * warp + q;
          q2v[q] = K0 + kk < G.ktot ? Qp[sm[kk].y + b] : 0.f;
        }
        for (int i = 0; i < na; ++i) {
          const float4 z0 = *reinterpret_cast<const float4*>(&zq1[i][8 * warp]);
          const float4 z1 = *reinterpret_cast<const float4*>(&zq1[i][8 * warp + 4]);
          float x[8] = {z0.x * q2v[0], z0.y * q2v[1], z0.z * q2v[2], z0.w * q2v[3],
                        z1.x * q2v[4], z1.y * q2v[5], z1.z * q2v[6], z1.w * q2v[7]};
          uint4 hi, lo;
          split8_f16(x, hi, lo);
          const int rho = (a0 + i) * r2 + b;
          unsigned char* blk = W + ((unsigned long long)(rho >> 7) * wstride + cl) * KR_A;
          const uint32_t off = kmajor_offset(rho & (CT_M - 1), warp, CT_KC / 8);
          *(uint4*)(blk + off) = hi;
          *(uint4*)(blk + CT_A_HALF + off) = lo;
        }
      }
    } else {
      const uint32_t krb = kr_b(G.cn);
      for (int nl = 0; nl < G.nt; ++nl) {
        unsigned char* blk = B3 + ((unsigned long long)nl * wstride + cl) * krb;
        for (int task = tid; task < G.cn * 8; task += 256) {
          const int kg = task / G.cn, row = task - kg * G.cn;
          const int cc = nl * G.cn + row;
          float x[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int kk = 8 * kg + q;
            x[q] = (cc < r3 && K0 + kk < G.ktot) ? fB * Qp[sm[kk].z + cc] : 0.f;
          }
          uint4 hi, lo;
          split8_f16(x, hi, lo);
          const uint32_t off = kmajor_offset(row, kg, CT_KC / 8);
          *(uint4*)(blk + off) = hi;
          *(uint4*)(blk + krb / 2 + off) = lo;
        }
      }
      const int first = pairs - (G.mt - 1) * CT_M;    // live rows of the last pair tile
      unsigned char* blk = W + ((unsigned long long)(G.mt - 1) * wstride + cl) * KR_A;
      for (int e = tid; e < (CT_M - first) * 8; e += 256) {
        const uint32_t off = kmajor_offset(first + (e >> 3), e & 7, CT_KC / 8);
        *(uint4*)(blk + off) = make_uint4(0u, 0u, 0u, 0u);
        *(uint4*)(blk + CT_A_HALF + off) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }
}

// x 2^e as a 64-bit integer, rounded to nearest (halves away from zero), from the bits of x
// with integer operations only; |x| 2^e < 2^63 (the fixed-point scale guarantees it)
__device__ __forceinline__ long long fx_f32(float x, int e) {
  const uint32_t u = __float_as_uint(x);
  const int ex = (int)((u >> 23) & 0xFFu);
  long long m = (long long)(u & 0x7FFFFFu);
  int s = e - 149;                                     // subnormal: x = m 2^-149
  if (ex != 0) {
    m |= 0x800000ll;
    s = ex - 150 + e;
  }
  long long r = 0;
  if (s >= 0)
    r = m << min(s, 39);
  else if (s > -26)
    r = (m + (1ll << (-s - 1))) >> (-s);
  return (u >> 31) ? -r : r;
}

struct KrArgs {
  const unsigned char* W;
  const unsigned char* B3;
  DevScalars* sc;
  double* beta64;
  int rmax, R_l, passes, pass, wstride;
};

template <int CN>
__device__ __forceinline__ void kr_body(const KrArgs& g, const KrGeom& G, unsigned char* smem) {
  // c tiles of CN values: stages of one A block and one B block, CN / 2 columns per epilogue warp
  constexpr uint32_t KRB = kr_b(CN);
  constexpr uint32_t KR_STAGE = KR_A + KRB;
  constexpr int KR_ST = (int)(KR_SMEM / KR_STAGE);
  constexpr int CH = CN / 2;
  __shared__ __align__(8) uint64_t bar_full[KR_ST], bar_empty[KR_ST];
  __shared__ __align__(8) uint64_t bar_dfull[2], bar_dempty[2], bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_s;
  volatile int* abort_flag = &abort_s;
  DevScalars* sc = g.sc;
  const long long c0 = (long long)g.pass * G.w;
  const int wl = (int)max(0ll, min((long long)G.w, G.kc - c0));
  const int tiles = G.mt * G.nt;
  // the (tile, chunk) pairs of the window, tile-major, split evenly over the CTAs; a CTA's range
  // falls into work units (one tile, consecutive chunks), each flushed to beta at its end
  const long long total = (long long)tiles * wl;
  const long long lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
  if (lo >= hi) return;                                // whole CTA, before any set-up
  auto next_unit = [&](long long pos, int& m, int& nl, int& cb, int& ce) -> long long {
    const int t = (int)(pos / wl);
    const long long end = min(hi, (long long)(t + 1) * wl);
    m = t / G.nt;
    nl = t - m * G.nt;
    cb = (int)(pos - (long long)t * wl);
    ce = cb + (int)(end - pos);
    return end;
  };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r1 = sc->rank[0], r2 = sc->rank[1], r3 = sc->rank[2];
  int sA, sB;
  kr_scales(sc, sA, sB);

  if (tid == 0) {
    for (int s = 0; s < KR_ST; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_dfull[b], 1);
      mbar_init(&bar_dempty[b], KR_EPI);
    }
    mbar_init(&bar_drain, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(KR_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint64_t dA = smem_desc(smem_addr(smem), 128, (CT_KC / 8) * 128);
      const uint64_t dB = smem_desc(smem_addr(smem + KR_A), 128, (CT_KC / 8) * 128);
      const uint64_t st_step = (uint64_t)KR_STAGE >> 4;
      const uint64_t a_lo = (uint64_t)CT_A_HALF >> 4, b_lo = (uint64_t)(KRB / 2) >> 4;
      const uint32_t idesc = idesc_f16(CN, CT_M);
      long long gc = 0, gseg = 0;
      bool ok = true;
      for (long long pos = lo; ok && pos < hi;) {
        int m, nl, cb, ce;
        pos = next_unit(pos, m, nl, cb, ce);
        for (int cl = cb; cl < ce; ++cl) {
          const int buf = (int)(gseg & 1);
          if (gseg >= 2 && !wait_bar(&bar_dempty[buf], (uint32_t)((gseg - 2) >> 1) & 1u, abort_flag, sc)) {
            ok = false;
            break;
          }
          const int st = (int)(gc % KR_ST);
          if (!wait_bar(&bar_full[st], (uint32_t)(gc / KR_ST) & 1u, abort_flag, sc)) {
            ok = false;
            break;
          }
          fence_after_sync();
          const uint32_t d = tmem + (uint32_t)(buf * CN);
          const uint64_t ah = dA + (uint64_t)st * st_step, al = ah + a_lo;
          const uint64_t bh = dB + (uint64_t)st * st_step, bl = bh + b_lo;
#pragma unroll
          for (int s4 = 0; s4 < CT_KC / 16; ++s4) {
            const uint64_t ko = (uint64_t)s4 * 16u;        // 16 FP16 = 32 bytes per row = 2 chunks
            mma_f16(d, ah + ko, bh + ko, idesc, s4 == 0 ? 0u : 1u);
            mma_f16(d, ah + ko, bl + ko, idesc, 1u);
            mma_f16(d, al + ko, bh + ko, idesc, 1u);
          }
          mma_commit(&bar_empty[st]);
          mma_commit(&bar_dfull[buf]);
          ++gc;
          ++gseg;
        }
      }
      // every MMA of this thread has completed before the tensor memory is released
      mma_commit(&bar_drain);
      drain_bar(&bar_drain, 0, sc);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ loader: bulk copies
    if (lane == 0) {
      long long gc = 0;
      bool ok = true;
      for (long long pos = lo; ok && pos < hi;) {
        int m, nl, cb, ce;
        pos = next_unit(pos, m, nl, cb, ce);
        for (int cl = cb; cl < ce; ++cl) {
          const int st = (int)(gc % KR_ST);
          if (gc >= KR_ST && !wait_bar(&bar_empty[st], (uint32_t)(gc / KR_ST - 1) & 1u, abort_flag, sc)) {
            ok = false;
            break;
          }
          unsigned char* base = smem + (size_t)st * KR_STAGE;
          mbar_expect_tx(&bar_full[st], KR_A + KRB);
          bulk_load(base, g.W + ((unsigned long long)m * g.wstride + cl) * KR_A, KR_A, &bar_full[st]);
          bulk_load(base + KR_A, g.B3 + ((unsigned long long)nl * g.wstride + cl) * KRB, KRB, &bar_full[st]);
          ++gc;
        }
      }
      // the copies issued last have landed before the shared memory goes away
      for (long long t = gc > KR_ST ? gc - KR_ST : 0; t < gc; ++t)
        drain_bar(&bar_full[t % KR_ST], (uint32_t)(t / KR_ST) & 1u, sc);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;                         // 0 .. 7
    const int q = warp & 3;                          // tensor-memory lanes 32q .. 32q + 31
    const int half = ew >> 2;                        // columns CH half .. CH half + CH - 1
    const int fx_e = beta_fx_shift(sc, g.R_l) - sA - sB;   // fixed-point exponent of the sums
    long long gseg = 0;
    bool ok = true;
    for (long long pos = lo; ok && pos < hi;) {
      int m, nl, cb, ce;
      pos = next_unit(pos, m, nl, cb, ce);
      float hi[CH], lo[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        hi[j] = 0.f;
        lo[j] = 0.f;
      }
      for (int cl = cb; cl < ce; ++cl) {
        const int buf = (int)(gseg & 1);
        if (!warp_wait(&bar_dfull[buf], (uint32_t)(gseg >> 1) & 1u, abort_flag, sc)) {
          ok = false;
          break;
        }
        fence_after_sync();
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * CN + CH * half);
        uint32_t v[CH];
#pragma unroll
        for (int u8 = 0; u8 < CH / 8; ++u8) tmem_ld8(ta + (uint32_t)(8 * u8), v + 8 * u8);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < CH; ++j) two_sum_acc(hi[j], lo[j], __uint_as_float(v[j]));
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_dempty[buf]);
        ++gseg;
      }
      if (!ok) break;
      const int rho = m * CT_M + 32 * q + lane;
      const int cbase = nl * CN + CH * half;
      if (rho < r1 * r2) {
        const int a = rho / r2, b = rho - a * r2;
        unsigned long long* out = reinterpret_cast<unsigned long long*>(g.beta64) +
                                  ((long long)a * g.rmax + b) * g.rmax + cbase;
#pragma unroll
        for (int j = 0; j < CH; ++j)
          if (cbase + j < r3) atomicAdd(out + j, (unsigned long long)(fx_f32(hi[j], fx_e) + fx_f32(lo[j], fx_e)));
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(KR_TMEM_COLS)
                 : "memory");
  }
}

__global__ void __launch_bounds__(KR_THREADS, 1) core_kr_kernel(KrArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const KrGeom G = kr_geom(g.sc, g.R_l, g.passes);
  if (G.cn == 64)
    kr_body<64>(g, G, smem);
  else
    kr_body<96>(g, G, smem);
}

// Workspace of the Khatri-Rao contraction for the context's rank cap and particle capacity:
// windows of at most `wstride` chunks, `passes` of them; 0 when it would take more than
// KR_MAX_PASSES windows (the contraction is then left to the other two forms).
size_t core_kr_plan(const Ctx& c, int& passes, int& wstride) {
  const long long mt = ((long long)c.rmax * c.rmax + CT_M - 1) / CT_M;
  const long long kc = ((long long)c.maxN * c.R_l + CT_KC - 1) / CT_KC;
  // q3 blocks for the wider of the two c tilings the ranks may choose
  const size_t b3 = std::max<size_t>((size_t)((c.rmax + 63) / 64) * kr_b(64), (size_t)((c.rmax + 95) / 96) * kr_b(96));
  const size_t per_chunk = (size_t)mt * KR_A + b3;
  const size_t grid_bytes = (size_t)4 * c.n * c.n * c.n;
  const size_t budget = std::max<size_t>((size_t)256 << 20, 2 * grid_bytes);
  long long p = (long long)(((size_t)kc * per_chunk + budget - 1) / budget);
  if (p < 1) p = 1;
  passes = (int)std::min<long long>(p, KR_MAX_PASSES + 1);
  wstride = (int)((kc + p - 1) / p);
  if (p > KR_MAX_PASSES || kc == 0) return 0;
  return per_chunk * (size_t)wstride;
}

int launch_core_kr(Ctx& c) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  const long long Kmax = (long long)c.maxN * c.R_l;
  const int mblocks = (int)((Kmax + 255) / 256);
  core_meta_kernel<<<mblocks > 0 ? mblocks : 1, 256, 0, c.stream>>>(c.j, c.nz_idx, c.Z, c.n, c.rmax, c.R_l, c.sc,
                                                                     (int4*)c.kmeta);
  const long long mt_max = ((long long)c.rmax * c.rmax + CT_M - 1) / CT_M;
  unsigned char* W = (unsigned char*)c.kr_buf;
  unsigned char* B3 = W + (size_t)mt_max * c.kr_wstride * KR_A;
  KrArgs g;
  g.W = W;
  g.B3 = B3;
  g.sc = c.sc;
  g.beta64 = c.beta64;
  g.rmax = c.rmax;
  g.R_l = c.R_l;
  g.passes = c.kr_passes;
  g.wstride = c.kr_wstride;
  for (int p = 0; p < c.kr_passes; ++p) {
    core_w_kernel<<<4 * sms, 256, 0, c.stream>>>((const float*)c.Qp, (const int4*)c.kmeta, c.sc, c.R_l,
                                                 c.kr_passes, p, c.kr_wstride, W, B3);
    g.pass = p;
    core_kr_kernel<<<sms, KR_THREADS, CT_SMEM, c.stream>>>(g);
  }
  return 1 + 2 * c.kr_passes;
}

int launch_core_tc(Ctx& c) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long Kmax = (long long)c.maxN * c.R_l;
  const int mblocks = (int)((Kmax + 255) / 256);
  core_meta_kernel<<<mblocks > 0 ? mblocks : 1, 256, 0, c.stream>>>(c.j, c.nz_idx, c.Z, c.n, c.rmax, c.R_l, c.sc,
                                                                     (int4*)c.kmeta);
  CoreArgs g;
  g.Qp = (const float*)c.Qp;
  g.meta = (const int4*)c.kmeta;
  g.sc = c.sc;
  g.beta64 = c.beta64;
  g.rmax = c.rmax;
  g.R_l = c.R_l;
  core_tc_kernel<<<sms > 0 ? sms : 1, CT_THREADS, CT_SMEM, c.stream>>>(g);
  return 2;
}

cudaError_t set_attributes_core(int optin) {
  (void)optin;
  cudaError_t e = cudaFuncSetAttribute((const void*)core_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)CT_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)core_kr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT_SMEM);
  return e;
}

}  // namespace rs
