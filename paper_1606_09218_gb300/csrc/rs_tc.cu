// Tensor-core (tcgen05) assembly of the FP32 RS potential on the grid.  One GEMM per output
// tile with a data-dependent K:
//
//   P[i1][i2][i3] = sum_a V1[i1][a] T2[a][i2][i3]                        Tucker part (Def. 3.9,
//                                                                         Eq. (3.11); Eq. (2.3))
//                 + sum_{nu in L(i)} sum_{k short} (z_nu p_k[i2-j2] p_k[i3-j3]) p_k[i1-j1]
//                                                                         windows (Defs. 3.4, 3.6)
//
// M = 128 grid points (i2, i3) of a 4 x 32 tile, N = a chunk of i1 rows, K = the Tucker rank r1
// followed by ceil8(R_s) per window that reaches the tile (each window is a rank-R_s outer
// product, so it is one more K slice of the same accumulator).  The accumulator lives in tensor
// memory, the sum is stored once, and the output is never read back: the Tucker product and
// the short-range windows cost one pass over the grid.
//
// Precision: every FP32 operand is split into a TF32 high part and a TF32 low part
// (x = hi + lo, |lo| <= 2^-11 |x|) and D += A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates in FP32
// (three tcgen05.mma kind::tf32 per K slice), an error of order 2^-21 |A||B| per product.
//
// CTA (persistent, one per SM, 14 warps):
//   warp 0     tensor-memory owner; lane 0 issues the MMAs
//   warp 1     scheduler: TMA load of the T2 slab of the next tile, window list pages
//   warps 2-5  producers: split T2 slab -> A (K-major, hi/lo); window operands -> slot ring
//   warps 6-13 epilogue: tensor memory -> registers -> coalesced streaming stores
// A CTA keeps one i1 chunk (its V1 rows, split, as the B operand of the Tucker part) and walks
// over the tiles; the accumulator is double-buffered so that the stores of one tile overlap the
// MMAs of the next.  Every wait is bounded: on expiry the CTA sets FLAG_TIMEOUT, the other roles
// see an abort flag, the MMA issuer and the TMA issuer wait (bounded) for their work in flight,
// and the tensor memory is released before return.
#include "rs_internal.cuh"

#include <cudaTypedefs.h>

#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace rs {

namespace {

constexpr int AS_M = 128;                  // grid points per tile (tensor-memory lanes)
constexpr int AS_T2 = 4, AS_T3 = 32;       // tile = 4 (i2) x 32 (i3)
constexpr int AS_THREADS = 448;            // 14 warps
constexpr int WARP_SCHED = 1, WARP_PROD = 2, WARP_EPI = 6;
constexpr int NPROD = 128;                 // producer threads
constexpr int NEPI = 8;                    // epilogue warps
constexpr int LIST_CAP = 256;              // window records per list page
constexpr int WL_SORT_CAP = 4096;          // longest window list of one tile column
constexpr long long WAIT_LIMIT = 4000000;
constexpr int SMEM_LIMIT = 232448;         // opt-in shared memory per CTA on this GPU family
constexpr int SMEM_RESERVE = 1024;         // static shared memory of the kernel

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

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
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

// Bounded wait for the phase with the given parity.  Returns false when another role has
// aborted or when the limit ran out (then this thread raises the abort and FLAG_TIMEOUT).
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         DevScalars* sc) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicOr(&sc->flags, (unsigned)FLAG_TIMEOUT);
  return false;
}

// Bounded wait that ignores the abort flag (draining work in flight before exit).
__device__ __forceinline__ void drain_bar(uint64_t* bar, uint32_t parity, DevScalars* sc) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_test(bar, parity)) return;
  atomicOr(&sc->flags, (unsigned)FLAG_TIMEOUT);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// canonical K-major layout without swizzle: 8-row x 16-byte core matrices, the K chunks of a
// row group contiguous (LBO = 128 B), row groups SBO = (kw/4)*128 B apart (kw = K width).
__device__ __forceinline__ uint32_t kmajor_offset(int row, int k4, int kw) {
  return ((uint32_t)(row >> 3) * (uint32_t)(kw >> 2) + (uint32_t)k4) * 128u + (uint32_t)(row & 7) * 16u;
}

// split four FP32 values into TF32 hi / lo and store both 16-byte chunks
__device__ __forceinline__ void store_split4(unsigned char* hi, unsigned char* lo, uint32_t off,
                                             float x0, float x1, float x2, float x3) {
  uint32_t h0 = to_tf32(x0), h1 = to_tf32(x1), h2 = to_tf32(x2), h3 = to_tf32(x3);
  uint32_t l0 = to_tf32(x0 - __uint_as_float(h0)), l1 = to_tf32(x1 - __uint_as_float(h1));
  uint32_t l2 = to_tf32(x2 - __uint_as_float(h2)), l3 = to_tf32(x3 - __uint_as_float(h3));
  *(uint4*)(hi + off) = make_uint4(h0, h1, h2, h3);
  *(uint4*)(lo + off) = make_uint4(l0, l1, l2, l3);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;      // leading dimension byte offset
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;      // stride dimension byte offset
  d |= (uint64_t)1 << 46;                            // fixed 0b001
  return d;                                           // base offset 0, no swizzle
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = nn
__device__ __forceinline__ uint32_t idesc_tf32(int nn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nn >> 3) << 17) | ((uint32_t)(AS_M >> 4) << 24);
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

// D (+)= A_hi B_hi + A_hi B_lo + A_lo B_hi for one K slice of 8
__device__ __forceinline__ void mma3(uint32_t d, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl,
                                     uint32_t sbo_a, uint32_t sbo_b, uint32_t idesc, uint32_t acc) {
  const uint64_t dah = smem_desc(ah, 128, sbo_a), dal = smem_desc(al, 128, sbo_a);
  const uint64_t dbh = smem_desc(bh, 128, sbo_b), dbl = smem_desc(bl, 128, sbo_b);
  mma_tf32(d, dah, dbh, idesc, acc);
  mma_tf32(d, dah, dbl, idesc, 1u);
  mma_tf32(d, dal, dbh, idesc, 1u);
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

// 8 consecutive accumulator columns of this warp's 32 lanes (one row per lane)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct AsmArgs {
  const float* V1;           // mode-1 Tucker basis, n x ldv
  int ldv;
  const float* pk;           // factor table, R x L (FP32)
  const int4* rec;           // window records (j1, j2, j3, float bits of z), per tile column
  const int2* rng;           // [tile][chunk] ranges into rec (nullptr: no short-range terms)
  float* P;                  // output n^3
  DevScalars* sc;
  int n, L, R_l, R_s;
  int nch, Nc, kpad, K8, gcap, nt3, ntiles, dstride, tmem_cols;
  uint32_t off_bh, off_bl, off_raw, off_ah, off_al, off_slot, slot_bytes, off_tab, off_list;
};

}  // namespace

__global__ void __launch_bounds__(AS_THREADS, 1)
assemble_kernel(const __grid_constant__ CUtensorMap tmap, const AsmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_raw_full, bar_raw_empty, bar_a_full, bar_a_free, bar_drain;
  __shared__ __align__(8) uint64_t bar_list_full[2], bar_list_empty[2];
  __shared__ __align__(8) uint64_t bar_slot_full[2], bar_slot_free[2];
  __shared__ __align__(8) uint64_t bar_d_full[2], bar_d_empty[2];
  __shared__ int page_n[2], page_total[2], job_nw[2], slot_hdr[2][2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_s;
  volatile int* abort_flag = &abort_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  DevScalars* sc = g.sc;
  const int n = g.n;
  const int chunk = (int)(blockIdx.x % (unsigned)g.nch);
  const int j0 = (int)(blockIdx.x / (unsigned)g.nch);
  const int jstride = (int)(gridDim.x / (unsigned)g.nch);
  const int c0 = chunk * g.Nc;
  const int cl = min(n, c0 + g.Nc) - 1;                 // last i1 row of this chunk
  const int r1 = sc->rank[0];
  const int gam = sc->gamma;
  const bool ok_gamma = gam <= g.gcap;
  const int njobs = (ok_gamma && j0 < g.ntiles && c0 < n) ? (g.ntiles - 1 - j0) / jstride + 1 : 0;
  const int tw = 2 * g.gcap + 1;                        // row length of the factor table
  const int kq = g.kpad >> 2;
  unsigned char* Bh = smem + g.off_bh;
  unsigned char* Bl = smem + g.off_bl;
  const float* raw = (const float*)(smem + g.off_raw);
  unsigned char* Ah = smem + g.off_ah;
  unsigned char* Al = smem + g.off_al;
  float* tab = (float*)(smem + g.off_tab);
  int4* lists = (int4*)(smem + g.off_list);

  if (tid == 0) {
    mbar_init(&bar_raw_full, 1);
    mbar_init(&bar_raw_empty, NPROD);
    mbar_init(&bar_a_full, NPROD);
    mbar_init(&bar_a_free, 1);
    mbar_init(&bar_drain, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_list_full[b], 1);
      mbar_init(&bar_list_empty[b], NPROD);
      mbar_init(&bar_slot_full[b], NPROD);
      mbar_init(&bar_slot_free[b], 1);
      mbar_init(&bar_d_full[b], 1);
      mbar_init(&bar_d_empty[b], NEPI);
    }
    abort_s = 0;
    if (!ok_gamma) atomicOr(&sc->flags, (unsigned)FLAG_WINDOWS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(g.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // one-time staging by the whole CTA: the short-range factor rows p_k[d], |d| <= gamma, and
  // the V1 rows of this chunk as the B operand of the Tucker part (K-major, hi / lo)
  if (njobs > 0) {
    for (int e = tid; e < g.R_s * tw; e += AS_THREADS) {
      const int k = e / tw, d = e % tw - g.gcap;
      tab[e] = (d >= -gam && d <= gam) ? g.pk[(long long)(g.R_l + k) * g.L + (n - 1) + d] : 0.f;
    }
    for (int e = tid; e < g.Nc * kq; e += AS_THREADS) {
      const int r = e / kq, k4 = e % kq, i1 = c0 + r;
      float x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = 4 * k4 + q;
        x[q] = (i1 < n && a < r1) ? g.V1[(long long)i1 * g.ldv + a] : 0.f;
      }
      store_split4(Bh, Bl, kmajor_offset(r, k4, g.kpad), x[0], x[1], x[2], x[3]);
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
      const uint32_t sbo_t = (uint32_t)kq * 128u, sbo_w = (uint32_t)(g.K8 >> 2) * 128u;
      const uint32_t bh = smem_addr(Bh), bl = smem_addr(Bl), ah = smem_addr(Ah), al = smem_addr(Al);
      const uint32_t slot0 = smem_addr(smem + g.off_slot);
      const uint32_t a_w = (uint32_t)AS_M * g.K8 * 4, b_w = (uint32_t)g.Nc * g.K8 * 4;
      const int ksteps = max(1, min(g.kpad, (r1 + 7) & ~7) >> 3);
      const uint32_t id_main = idesc_tf32(g.Nc);
      int gw = 0;
      for (int t = 0; t < njobs; ++t) {
        if (!wait_bar(&bar_a_full, t & 1, abort_flag, sc)) break;
        const int nw = job_nw[t & 1];
        if (t >= 2 && !wait_bar(&bar_d_empty[t & 1], ((t - 2) >> 1) & 1, abort_flag, sc)) break;
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)((t & 1) * g.dstride);
        for (int s = 0; s < ksteps; ++s) {
          const uint32_t ko = (uint32_t)s * 256u;   // two 16-byte K chunks per slice of 8
          mma3(d, ah + ko, al + ko, bh + ko, bl + ko, sbo_t, sbo_t, id_main, s > 0 ? 1u : 0u);
        }
        mma_commit(&bar_a_free);
        bool ok = true;
        for (int w = 0; w < nw; ++w, ++gw) {
          const int s = gw & 1;
          if (!wait_bar(&bar_slot_full[s], (gw >> 1) & 1, abort_flag, sc)) { ok = false; break; }
          fence_after_sync();
          const int s0 = slot_hdr[s][0], s1 = slot_hdr[s][1];
          const uint32_t base = slot0 + (uint32_t)s * g.slot_bytes;
          const uint32_t wah = base, wal = base + a_w, wbh = base + 2 * a_w, wbl = base + 2 * a_w + b_w;
          const uint32_t boff = (uint32_t)s0 * 2u * sbo_w;          // 16 rows = 2 row groups
          const uint32_t id_w = idesc_tf32(16 * (s1 - s0 + 1));
          const uint32_t dw = d + (uint32_t)(16 * s0);
          for (int ks = 0; ks < (g.K8 >> 3); ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
            mma3(dw, wah + ko, wal + ko, wbh + boff + ko, wbl + boff + ko, sbo_w, sbo_w, id_w, 1u);
          }
          mma_commit(&bar_slot_free[s]);
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
    int pg = 0, issued = 0;
    for (int t = 0; t < njobs; ++t) {
      const int T = j0 + t * jstride, t2 = T / g.nt3, t3 = T % g.nt3;
      int ok = 1;
      if (lane == 0) {
        if (t > 0) ok = wait_bar(&bar_raw_empty, (t - 1) & 1, abort_flag, sc);
        if (ok) {
          mbar_expect_tx(&bar_raw_full, (uint32_t)(AS_M * g.kpad * 4));
          tma_load_3d(smem + g.off_raw, &tmap, t3 * AS_T3, t2 * AS_T2, 0, &bar_raw_full);
          ++issued;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      int2 rg = make_int2(0, 0);
      if (g.rng) rg = g.rng[(long long)T * g.nch + chunk];
      const int total = rg.y - rg.x;
      for (int off = 0;; off += LIST_CAP) {
        const int b = pg & 1;
        if (lane == 0 && pg >= 2) ok = wait_bar(&bar_list_empty[b], ((pg - 2) >> 1) & 1, abort_flag, sc);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        const int cnt = min(LIST_CAP, total - off);
        for (int i = lane; i < cnt; i += 32) lists[b * LIST_CAP + i] = g.rec[rg.x + off + i];
        if (lane == 0) { page_n[b] = cnt; page_total[b] = total; }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_list_full[b]);
        ++pg;
        if (off + LIST_CAP >= total) break;
      }
      if (!ok) break;
    }
    // the last TMA load has landed before the CTA exits
    if (lane == 0 && issued > 0) drain_bar(&bar_raw_full, (issued - 1) & 1, sc);
    __syncwarp();
  } else if (warp < WARP_EPI) {
    // ------------------------------------------------------------ producers
    const int pt = tid - WARP_PROD * 32;
    const int kw = g.K8;
    unsigned char* slot_base = smem + g.off_slot;
    const uint32_t a_w = (uint32_t)AS_M * kw * 4, b_w = (uint32_t)g.Nc * kw * 4;
    int pg = 0, gw = 0;
    for (int t = 0; t < njobs; ++t) {
      const int T = j0 + t * jstride, t2 = T / g.nt3, t3 = T % g.nt3;
      int b = pg & 1;
      if (!wait_bar(&bar_raw_full, t & 1, abort_flag, sc)) break;
      if (!wait_bar(&bar_list_full[b], (pg >> 1) & 1, abort_flag, sc)) break;
      if (t > 0 && !wait_bar(&bar_a_free, (t - 1) & 1, abort_flag, sc)) break;
      // T2 slab (a, m) -> A rows m, K-major, hi / lo; ranks beyond r1 are zero
      for (int k4 = 0; k4 < kq; ++k4) {
        float x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int a = 4 * k4 + q;
          x[q] = (a < r1) ? raw[a * AS_M + pt] : 0.f;
        }
        store_split4(Ah, Al, kmajor_offset(pt, k4, g.kpad), x[0], x[1], x[2], x[3]);
      }
      const int nw = page_total[b];
      if (pt == 0) job_nw[t & 1] = nw;
      fence_proxy_async();
      mbar_arrive(&bar_a_full);
      mbar_arrive(&bar_raw_empty);
      // windows: A_w[m][k] = z p_k[i2-j2] p_k[i3-j3],  B_w[i1][k] = p_k[i1-j1]
      const int i2 = t2 * AS_T2 + (pt >> 5), i3 = t3 * AS_T3 + (pt & 31);
      const int i1 = c0 + pt;
      bool ok = true;
      int pos = 0, pn = page_n[b];
      for (int w = 0; w < nw; ++w, ++gw) {
        if (pos == pn) {
          mbar_arrive(&bar_list_empty[b]);
          ++pg;
          b = pg & 1;
          if (!wait_bar(&bar_list_full[b], (pg >> 1) & 1, abort_flag, sc)) { ok = false; break; }
          pos = 0;
          pn = page_n[b];
        }
        const int4 rc = lists[b * LIST_CAP + pos];
        ++pos;
        const int s = gw & 1;
        if (gw >= 2 && !wait_bar(&bar_slot_free[s], ((gw - 2) >> 1) & 1, abort_flag, sc)) { ok = false; break; }
        unsigned char* sb = slot_base + (size_t)s * g.slot_bytes;
        const float z = __int_as_float(rc.w);
        const int d2 = i2 - rc.y, d3 = i3 - rc.z, d1 = i1 - rc.x;
        const bool in23 = i2 < n && i3 < n && d2 >= -gam && d2 <= gam && d3 >= -gam && d3 <= gam;
        const float* t2row = tab + (d2 + g.gcap);
        const float* t3row = tab + (d3 + g.gcap);
        for (int k4 = 0; k4 < (kw >> 2); ++k4) {
          float x[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int k = 4 * k4 + q;
            x[q] = (in23 && k < g.R_s) ? z * t2row[k * tw] * t3row[k * tw] : 0.f;
          }
          store_split4(sb, sb + a_w, kmajor_offset(pt, k4, kw), x[0], x[1], x[2], x[3]);
        }
        if (pt < g.Nc) {
          const bool in1 = i1 < n && d1 >= -gam && d1 <= gam;
          const float* t1row = tab + (d1 + g.gcap);
          for (int k4 = 0; k4 < (kw >> 2); ++k4) {
            float x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int k = 4 * k4 + q;
              x[q] = (in1 && k < g.R_s) ? t1row[k * tw] : 0.f;
            }
            store_split4(sb + 2 * a_w, sb + 2 * a_w + b_w, kmajor_offset(pt, k4, kw), x[0], x[1],
                         x[2], x[3]);
          }
        }
        if (pt == 0) {
          // 16-column groups of the chunk that this window reaches
          const int lo1 = max(c0, rc.x - gam) - c0, hi1 = min(cl, rc.x + gam) - c0;
          slot_hdr[s][0] = lo1 >> 4;
          slot_hdr[s][1] = hi1 >> 4;
        }
        fence_proxy_async();
        mbar_arrive(&bar_slot_full[s]);
      }
      if (!ok) break;
      mbar_arrive(&bar_list_empty[b]);
      ++pg;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - WARP_EPI;
    const int q = warp & 3;                        // tensor-memory lanes 32q .. 32q+31
    const int half = ew >> 2;
    const int cb = half * (g.Nc >> 1), ce = cb + (g.Nc >> 1);
    const long long plane = (long long)n * n;
    for (int t = 0; t < njobs; ++t) {
      const int T = j0 + t * jstride, t2 = T / g.nt3, t3 = T % g.nt3;
      int ok = 1;
      if (lane == 0) ok = wait_bar(&bar_d_full[t & 1], (t >> 1) & 1, abort_flag, sc);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      fence_after_sync();
      const int i2 = t2 * AS_T2 + q, i3 = t3 * AS_T3 + lane;
      const bool valid = i2 < n && i3 < n;
      float* out = g.P + (long long)i2 * n + i3;
      const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((t & 1) * g.dstride);
      for (int c = cb; c < ce; c += 32) {
        uint32_t v[32];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (c + 8 * u < ce) tmem_ld8(base + (uint32_t)(c + 8 * u), v + 8 * u);
        tmem_wait_ld();
        if (valid) {
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const int i1 = c0 + c + u;
            if (c + u < ce && i1 < n) __stcs(out + (long long)i1 * plane, __uint_as_float(v[u]));
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_d_empty[t & 1]);
    }
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
// For every output tile column (4 i2 x 32 i3 points, all i1) the particles whose window
// (|i_l - j_l| <= gamma) reaches it, sorted by (j1, particle) so that the windows of one i1
// chunk are a contiguous range and the summation order does not depend on scheduling.
__global__ void wl_count_kernel(const int* __restrict__ jidx, const int* __restrict__ nz_idx,
                                const DevScalars* sc, int n, int nt3, int* count) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= sc->n_nz) return;
  const int p = nz_idx[m], g = sc->gamma;
  const int j2 = jidx[3 * p + 1], j3 = jidx[3 * p + 2];
  const int a2 = max(0, j2 - g) / AS_T2, b2 = min(n - 1, j2 + g) / AS_T2;
  const int a3 = max(0, j3 - g) / AS_T3, b3 = min(n - 1, j3 + g) / AS_T3;
  for (int t2 = a2; t2 <= b2; ++t2)
    for (int t3 = a3; t3 <= b3; ++t3) atomicAdd(&count[t2 * nt3 + t3], 1);
}

__global__ void wl_fill_kernel(const int* __restrict__ jidx, const int* __restrict__ nz_idx,
                               DevScalars* sc, int n, int nt3, const int* start, int* cursor,
                               long long cap, long long* key) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= sc->n_nz) return;
  const int p = nz_idx[m], g = sc->gamma;
  const int j1 = jidx[3 * p], j2 = jidx[3 * p + 1], j3 = jidx[3 * p + 2];
  const int a2 = max(0, j2 - g) / AS_T2, b2 = min(n - 1, j2 + g) / AS_T2;
  const int a3 = max(0, j3 - g) / AS_T3, b3 = min(n - 1, j3 + g) / AS_T3;
  const long long k = ((long long)j1 << 32) | (unsigned)p;
  for (int t2 = a2; t2 <= b2; ++t2)
    for (int t3 = a3; t3 <= b3; ++t3) {
      const int T = t2 * nt3 + t3;
      const long long pos = (long long)start[T] + atomicAdd(&cursor[T], 1);
      if (pos < cap) key[pos] = k;
      else atomicOr(&sc->flags, (unsigned)FLAG_WINDOWS);
    }
}

// one CTA per tile column: bitonic sort of its keys, records, and the range of each i1 chunk
__global__ void __launch_bounds__(256)
wl_sort_kernel(const int* __restrict__ start, long long cap, const long long* __restrict__ key,
               const int* __restrict__ jidx, const double* __restrict__ Z, DevScalars* sc, int n,
               int nch, int Nc, int4* rec, int2* rng) {
  __shared__ long long ks[WL_SORT_CAP];
  const int T = blockIdx.x, tid = threadIdx.x;
  const long long s = min((long long)start[T], cap), e = min((long long)start[T + 1], cap);
  int len = (int)(e - s);
  const int g = sc->gamma;
  if (len > WL_SORT_CAP) {
    if (tid == 0) atomicOr(&sc->flags, (unsigned)FLAG_WINDOWS);
    for (int c = tid; c < nch; c += blockDim.x) rng[(long long)T * nch + c] = make_int2((int)s, (int)s);
    return;
  }
  int m = 1;
  while (m < len) m <<= 1;
  for (int i = tid; i < m; i += blockDim.x) ks[i] = (i < len) ? key[s + i] : LLONG_MAX;
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1)
    for (int jx = k >> 1; jx > 0; jx >>= 1) {
      for (int i = tid; i < m; i += blockDim.x) {
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
    int lo2 = lo, hi2 = len;                    // first key with j1 > hi_j
    while (lo2 < hi2) { const int mid = (lo2 + hi2) >> 1; if ((int)(ks[mid] >> 32) <= hi_j) lo2 = mid + 1; else hi2 = mid; }
    rng[(long long)T * nch + c] = make_int2((int)(s + lo), (int)(s + lo2));
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
  const int nT = c.tc_nt2 * c.tc_nt3;
  int grid = (c.maxN + 255) / 256;
  if (grid < 1) grid = 1;
  cudaMemsetAsync(c.wl_count, 0, sizeof(int) * (nT + 1), c.stream);
  wl_count_kernel<<<grid, 256, 0, c.stream>>>(c.j, c.nz_idx, c.sc, c.n, c.tc_nt3, c.wl_count);
  wl_scan_kernel<<<1, 1024, 0, c.stream>>>(c.wl_count, nT, c.wl_start);
  cudaMemsetAsync(c.wl_count, 0, sizeof(int) * (nT + 1), c.stream);
  wl_fill_kernel<<<grid, 256, 0, c.stream>>>(c.j, c.nz_idx, c.sc, c.n, c.tc_nt3, c.wl_start,
                                             c.wl_count, c.wl_cap, c.wl_key);
  wl_sort_kernel<<<nT, 256, 0, c.stream>>>(c.wl_start, c.wl_cap, c.wl_key, c.j, c.Z, c.sc, c.n,
                                           c.tc_nch, c.tc_Nc, c.wl_rec, c.wl_rng);
  return 4;
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

}  // namespace

bool plan_assemble(Ctx& c) {
  if (c.fp64) return false;
  const char* env = std::getenv("RS_RECON_PATH");
  if (env && std::strcmp(env, "cuda") == 0) return false;
  const int n = c.n;
  const int gh = host_gamma(c);
  c.gamma_cap = gh + 1 < n - 1 ? gh + 1 : n - 1;
  c.tc_kpad = (c.rmax + 7) & ~7;
  c.tc_K8 = c.R_s > 8 ? 16 : 8;
  c.tc_nch = (n + 127) / 128;
  const int per = (n + c.tc_nch - 1) / c.tc_nch;
  c.tc_Nc = (per + 15) & ~15;
  c.tc_nt2 = (n + AS_T2 - 1) / AS_T2;
  c.tc_nt3 = (n + AS_T3 - 1) / AS_T3;
  if (c.tc_kpad > 256) return false;                       // TMA box extent
  const size_t sz_b = al128((size_t)c.tc_Nc * c.tc_kpad * 4);
  const size_t sz_a = al128((size_t)AS_M * c.tc_kpad * 4);
  const size_t slot = al128((size_t)2 * (AS_M + c.tc_Nc) * c.tc_K8 * 4);
  const size_t sz_tab = al128((size_t)c.R_s * (2 * c.gamma_cap + 1) * 4);
  const size_t total = 2 * sz_b + 3 * sz_a + 2 * slot + sz_tab + (size_t)2 * LIST_CAP * 16;
  if (total > (size_t)(SMEM_LIMIT - SMEM_RESERVE)) return false;
  c.tc_smem = total;
  const long long touch2 = std::min<long long>(c.tc_nt2, (2 * c.gamma_cap) / AS_T2 + 2);
  const long long touch3 = std::min<long long>(c.tc_nt3, (2 * c.gamma_cap) / AS_T3 + 2);
  long long cap = (long long)c.maxN * touch2 * touch3;
  if (cap < 1) cap = 1;
  if (cap > INT_MAX / 2) return false;
  c.wl_cap = cap;
  c.t2_ld = (n + 3) & ~3;
  return true;
}

bool encode_t2_map(Ctx& c, std::string& err) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    err = "cuTensorMapEncodeTiled not available";
    return false;
  }
  auto enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  const cuuint64_t dims[3] = {(cuuint64_t)c.n, (cuuint64_t)c.n, (cuuint64_t)c.rmax};
  const cuuint64_t strides[2] = {(cuuint64_t)c.t2_ld * 4, (cuuint64_t)c.n * c.t2_ld * 4};
  const cuuint32_t box[3] = {AS_T3, AS_T2, (cuuint32_t)c.tc_kpad};
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(&c.tmap_T2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c.T2, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled rejected the T2 view";
    return false;
  }
  return true;
}

int launch_assemble(Ctx& c, float* out) {
  AsmArgs g;
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
  g.kpad = c.tc_kpad;
  g.K8 = c.tc_K8;
  g.gcap = c.gamma_cap;
  g.nt3 = c.tc_nt3;
  g.ntiles = c.tc_nt2 * c.tc_nt3;
  int ds = 16;
  while (ds < c.tc_Nc) ds <<= 1;
  g.dstride = ds;
  g.tmem_cols = 2 * ds < 32 ? 32 : 2 * ds;
  const size_t sz_b = al128((size_t)c.tc_Nc * c.tc_kpad * 4);
  const size_t sz_a = al128((size_t)AS_M * c.tc_kpad * 4);
  const size_t slot = al128((size_t)2 * (AS_M + c.tc_Nc) * c.tc_K8 * 4);
  const size_t sz_tab = al128((size_t)c.R_s * (2 * c.gamma_cap + 1) * 4);
  g.off_bh = 0;
  g.off_bl = (uint32_t)sz_b;
  g.off_raw = (uint32_t)(2 * sz_b);
  g.off_ah = (uint32_t)(2 * sz_b + sz_a);
  g.off_al = (uint32_t)(2 * sz_b + 2 * sz_a);
  g.off_slot = (uint32_t)(2 * sz_b + 3 * sz_a);
  g.slot_bytes = (uint32_t)slot;
  g.off_tab = (uint32_t)(2 * sz_b + 3 * sz_a + 2 * slot);
  g.off_list = (uint32_t)(2 * sz_b + 3 * sz_a + 2 * slot + sz_tab);
  if (c.tc_grid == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    const int per_chunk = sms / c.tc_nch > 0 ? sms / c.tc_nch : 1;
    c.tc_grid = c.tc_nch * per_chunk;
    cudaFuncSetAttribute(assemble_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.tc_smem);
  }
  assemble_kernel<<<c.tc_grid, AS_THREADS, c.tc_smem, c.stream>>>(c.tmap_T2, g);
  return 1;
}

}  // namespace rs
