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
// this contraction is used where the Tucker tolerance is at least 1e-5 (1025^3 lattice: 2e-7
// of the oracle), and the CUDA-core contraction below that.
//
// Operand scales: A carries 2^sA with 2^sA max|z| max|q| < 2^14 and B 2^sB with
// 2^sB max|q|^2 < 2^14 (exact powers of two, removed when the units add to beta).
//
// CTA (one per SM, 16 warps):
//   warp 0      tensor-memory owner; lane 0 issues the MMAs into two accumulator buffers
//   warps 1-7   producers: A and B chunks of 64 K terms -> ring of four stages
//   warps 8-15  epilogue: a segment's accumulator -> (hi, lo) registers; FP64 atomics per unit
// Every wait is bounded (FLAG_TIMEOUT, abort flag, tensor memory released before return).
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
  return cudaFuncSetAttribute((const void*)core_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT_SMEM);
}

}  // namespace rs
