// Tensor-core (tcgen05) last mode product of the Tucker-to-full reconstruction
// (Def. 3.9, Eq. (3.11); Eq. (2.3)):
//     P[i1][p] = sum_a V1[i1][a] * T2[a][p],       p = (i2, i3) flattened,
// a GEMM with M = i1 (n rows), N = n^2 grid points, K = r1 (Tucker rank, <= 104).
//
// Precision: each FP32 operand is split into a TF32 high part and a TF32 low part
// (x = hi + lo, |lo| <= 2^-11 |x|) and D += A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in
// FP32 in tensor memory (three tcgen05.mma kind::tf32 per K step), leaving an error of order
// 2^-22 |A||B| per product.
//
// CTA layout (288 threads): warp 0 owns the tensor memory and one of its threads issues the
// MMAs, warps 1-4 produce operand tiles (load FP32, split, write the canonical no-swizzle
// K-major layout), warps 5-8 drain tensor memory (tcgen05.ld) and store the FP32 results.  One CTA owns BN grid points, keeps their T2 slab in
// shared memory and walks over the i1 tiles of 128 rows; the accumulator is double-buffered in
// tensor memory so that the store of one tile overlaps the MMAs of the next.  Every wait is
// bounded: on expiry the CTA sets FLAG_TIMEOUT, stops, releases its tensor memory and returns.
#include "rs_internal.cuh"

namespace rs {

namespace {

constexpr int TC_M = 128;              // rows of D per MMA (i1)
constexpr long long WAIT_LIMIT = 4000000;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity; false (and FLAG_TIMEOUT) on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevScalars* sc) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_test(bar, parity)) return true;
  atomicOr(&sc->flags, (unsigned)FLAG_TIMEOUT);
  return false;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// canonical K-major layout without swizzle: 8-row x 16-byte core matrices, the K chunks of a
// row group contiguous (LBO = 128 B), row groups SBO = (kpad/4)*128 B apart.
__device__ __forceinline__ uint32_t kmajor_offset(int row, int k4, int kpad) {
  return ((uint32_t)(row >> 3) * (uint32_t)(kpad >> 2) + (uint32_t)k4) * 128u + (uint32_t)(row & 7) * 16u;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;      // leading dimension byte offset
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;      // stride dimension byte offset
  d |= (uint64_t)1 << 46;                            // fixed 0b001
  return d;                                           // base offset 0, no swizzle
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// BN: grid points per CTA (256 or 128).  Dynamic shared memory: B_hi, B_lo (BN x kpad),
// A_hi, A_lo (128 x kpad).  Warps: 0 = tensor-memory owner and MMA issuer, 1-4 = producers,
// 5-8 = epilogue (warp w drains accumulator lanes 32*(w%4) .. 32*(w%4)+31).
constexpr int TC_THREADS = 288;
template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
recon_tc_kernel(const float* __restrict__ V1, int ldv, const float* __restrict__ T2, long long np,
                int n, int kpad, DevScalars* sc, float* __restrict__ P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full_b, bar_full_a, bar_mma[2], bar_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ float tr[4][32][33];             // per epilogue warp: 32 x 32 transpose tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r1 = sc->rank[0];
  const long long p0 = (long long)blockIdx.x * BN;
  const int ntile = (n + TC_M - 1) / TC_M;
  const uint32_t b_bytes = (uint32_t)BN * kpad * 4, a_bytes = (uint32_t)TC_M * kpad * 4;
  unsigned char* Bh = smem;
  unsigned char* Bl = smem + b_bytes;
  unsigned char* Ah = smem + 2 * b_bytes;
  unsigned char* Al = smem + 2 * b_bytes + a_bytes;

  if (tid == 0) {
    mbar_init(&bar_full_b, 128);
    mbar_init(&bar_full_a, 128);
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    mbar_init(&bar_empty[0], 128);
    mbar_init(&bar_empty[1], 128);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(2 * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                             ((uint32_t)(TC_M >> 4) << 24);
      const uint32_t lbo = 128, sbo = (uint32_t)(kpad >> 2) * 128u;
      const uint32_t bh = smem_addr(Bh), bl = smem_addr(Bl), ah = smem_addr(Ah), al = smem_addr(Al);
      bool ok = mbar_wait(&bar_full_b, 0, sc);
      for (int t = 0; ok && t < ntile; ++t) {
        // producers fill A for tile t only after the MMAs of tile t-1 completed, so the t-th
        // completion of bar_full_a has parity t & 1
        ok = mbar_wait(&bar_full_a, t & 1, sc);
        if (ok && t >= 2) ok = mbar_wait(&bar_empty[t & 1], ((t - 2) >> 1) & 1, sc);
        if (!ok) break;
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)((t & 1) * BN);
        for (int s = 0; s < (kpad >> 3); ++s) {
          const uint32_t ko = (uint32_t)s * 256u;     // two 16-byte K chunks per step
          const uint64_t dah = smem_desc(ah + ko, lbo, sbo), dal = smem_desc(al + ko, lbo, sbo);
          const uint64_t dbh = smem_desc(bh + ko, lbo, sbo), dbl = smem_desc(bl + ko, lbo, sbo);
          mma_tf32(d, dah, dbh, idesc, s > 0 ? 1u : 0u);
          mma_tf32(d, dah, dbl, idesc, 1u);
          mma_tf32(d, dal, dbh, idesc, 1u);
        }
        mma_commit(&bar_mma[t & 1]);
      }
    }
    __syncwarp();
  } else if (warp <= 4) {
    // ---------------- producers (128 threads): load FP32, split into TF32 hi/lo
    const int pt = tid - 32;
    for (int e = pt; e < BN * (kpad >> 2); e += 128) {
      const int nn = e % BN, k4 = e / BN;
      const long long p = p0 + nn;
      uint32_t h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = 4 * k4 + q;
        const float x = (p < np && a < r1) ? __ldg(T2 + (long long)a * np + p) : 0.f;
        h[q] = to_tf32(x);
        l[q] = to_tf32(x - __uint_as_float(h[q]));
      }
      const uint32_t off = kmajor_offset(nn, k4, kpad);
      *(uint4*)(Bh + off) = make_uint4(h[0], h[1], h[2], h[3]);
      *(uint4*)(Bl + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    fence_proxy_async();
    mbar_arrive(&bar_full_b);
    for (int t = 0; t < ntile; ++t) {
      if (t > 0 && !mbar_wait(&bar_mma[(t - 1) & 1], ((t - 1) >> 1) & 1, sc)) break;  // A is free
      for (int e = pt; e < TC_M * (kpad >> 2); e += 128) {
        const int rr = e / (kpad >> 2), k4 = e % (kpad >> 2);
        const int i1 = t * TC_M + rr;
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int a = 4 * k4 + q;
          const float x = (i1 < n && a < r1) ? __ldg(V1 + (long long)i1 * ldv + a) : 0.f;
          h[q] = to_tf32(x);
          l[q] = to_tf32(x - __uint_as_float(h[q]));
        }
        const uint32_t off = kmajor_offset(rr, k4, kpad);
        *(uint4*)(Ah + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *(uint4*)(Al + off) = make_uint4(l[0], l[1], l[2], l[3]);
      }
      fence_proxy_async();
      mbar_arrive(&bar_full_a);
    }
  } else {
    // ---------------- epilogue (warps 5-8): tensor memory -> registers -> smem transpose -> global
    const int q = warp & 3;                     // accumulator lanes 32q .. 32q+31
    float (*T)[33] = tr[q];
    for (int t = 0; t < ntile; ++t) {
      if (!mbar_wait(&bar_mma[t & 1], (t >> 1) & 1, sc)) break;
      fence_after_sync();
      const int row0 = t * TC_M + 32 * q;       // first i1 of this warp's 32 rows
      const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((t & 1) * BN);
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld32(base + (uint32_t)c0, v);     // this lane: row row0 + lane, columns c0..c0+31
#pragma unroll
        for (int j = 0; j < 32; ++j) T[lane][j] = v[j];
        __syncwarp();
        const long long p = p0 + c0 + lane;
        if (p < np) {
          for (int r = 0; r < 32; ++r) {
            const int i1 = row0 + r;
            if (i1 < n) P[(long long)i1 * np + p] = T[r][lane];
          }
        }
        __syncwarp();
      }
      fence_before_sync();
      mbar_arrive(&bar_empty[t & 1]);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN)
                 : "memory");
  }
}

// Returns the number of kernels launched, or -1 when the shape is not supported (the caller
// then uses the CUDA-core product).  Ranks are read on the device; kpad covers rmax.
int launch_recon_tc(Ctx& c, float* out) {
  const int n = c.n;
  const int kpad = ((c.rmax + 7) / 8) * 8;
  int bn;
  if (kpad <= 64) bn = 256;
  else if (kpad <= 104) bn = 128;
  else return -1;
  const long long np = (long long)n * n;
  const size_t shm = (size_t)2 * bn * kpad * 4 + (size_t)2 * 128 * kpad * 4;
  const unsigned grid = (unsigned)((np + bn - 1) / bn);
  const float* V1 = c.Z32;
  const float* T2 = (const float*)c.T2;
  if (bn == 256) {
    cudaFuncSetAttribute(recon_tc_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    recon_tc_kernel<256><<<grid, TC_THREADS, shm, c.stream>>>(V1, c.rmax, T2, np, n, kpad, c.sc, out);
  } else {
    cudaFuncSetAttribute(recon_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    recon_tc_kernel<128><<<grid, TC_THREADS, shm, c.stream>>>(V1, c.rmax, T2, np, n, kpad, c.sc, out);
  }
  return 1;
}

}  // namespace rs
