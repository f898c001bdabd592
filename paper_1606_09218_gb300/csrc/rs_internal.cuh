// Internal declarations of the RS library (CUDA path only).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>

#include "../../include/rs.h"

namespace rs {

// Width of the column blocks of the block Gram-Schmidt orthonormalisation.
constexpr int KB = 8;
// CTAs per mode of the cooperative block Gram-Schmidt kernel (3 x 48 = 144 <= 152 SMs).
constexpr int NBC = 48;
static_assert(NBC % 8 == 0, "the Gram-Schmidt reductions split the CTAs of a mode over 8 lanes");
// Largest Tucker rank the projection kernel supports.
constexpr int RMAX_LIMIT = 160;
// Largest subspace width the one-CTA Jacobi kernel holds in shared memory.
constexpr int KSUB_MAX = 160;
// Nonzeros per row of the sparse range-finder embedding.
constexpr int ZETA = 4;
// Side of the particle bins used to find the windows that touch a grid tile.
constexpr int BIN = 16;

// Device-side status bits (accumulated with atomicOr, read by rs_report).
enum : unsigned {
  FLAG_OUTSIDE = 1u,      // centre outside the box or non-finite input
  FLAG_SEPARATION = 2u,   // two centres closer than min_sep
  FLAG_RANK_CAPPED = 4u,  // eps not met within the rank limit
  FLAG_CHOL = 8u,         // a Cholesky factor of a Gram-Schmidt block was not positive
  FLAG_TIMEOUT = 16u,     // a bounded grid-barrier wait ran out
  FLAG_WINDOWS = 32u      // a window list outgrew its capacity (see the list builders)
};

// Scalars shared by the kernels of one solve (device memory).
struct DevScalars {
  // energy and flags first: rs_energy reads back only these 16 bytes
  double energy;
  unsigned flags;
  unsigned pad0;
  double P_R0, P_Rl0, delta;
  double zabs_sum;          // sum of |z| over the particles (bound of the core sums)
  unsigned long long w2max_bits;   // largest |z|^{2/3} (double bits; scale of the weight sums)
  double trG[3], trT[3], xnorm2[3], tail_rel[3];
  int gamma;
  int n_nz;                 // particles with nonzero charge
  int nzj_count[3];         // distinct grid coordinates carrying charge, per mode
  int k_eff[3];             // accepted Gram-Schmidt columns per mode
  int rank[3];              // Tucker ranks
  unsigned stopmask;             // modes whose Gram-Schmidt has finished
  int blk_acc[3];                // columns accepted by the one-CTA fallback of the current block
  int jacobi_sweeps;             // Jacobi sweeps of the last solve (all modes and passes)
  int fallbacks;                 // blocks that took the one-CTA Gram-Schmidt fallback
  int chunk_w[32];               // windows per i1 chunk (tensor-core assembly schedule)
  unsigned zmax_bits;            // max |z| over the particles (float bits; window operand scale)
  unsigned qmax_bits;            // max |Qp| of the FP32 projections (float bits; core operand scale)
  int t2_shift;                  // scale exponent S of the T2 tiles (written by the tile kernel)
  double beta_a2[RMAX_LIMIT];    // ||beta[a, :, :]||^2 (scale of the FP16 Tucker operands)
  // barriers of the cooperative Gram-Schmidt kernel, one per mode: arrival counter and
  // generation of mode l at [32 l], each on its own 128-byte line, so that the waiters' polling
  // does not slow the arrivals
  alignas(128) unsigned bar_count[3 * 32];
  alignas(128) unsigned bar_gen[3 * 32];
};

// scratch of the deterministic K split of the FP64 products: GEMM_SPLIT_SLOTS partial 16x16
// tiles and as many arrival counters (a split product has fewer than 2 x 152 tiles and at most
// ceil(2 x 152 / tiles) parts per tile, so fewer than 608 partials)
constexpr long long GEMM_SPLIT_SLOTS = 608;
struct GemmScratch {
  double* part = nullptr;
  unsigned* count = nullptr;
};

struct Ctx {
  rs_config cfg;
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;    // window lists and particle bins, overlapped with the eigen stage
  GemmScratch gscr;              // deterministic K split of the FP64 products
  // RS-canonical form of the last solve (allocated by the first rs_canonical call)
  double* cn_sig = nullptr;      // rmax x rmax singular values of the core slices
  double* cn_X = nullptr;        // rmax^3: left singular vectors per (slice, term)
  double* cn_Y = nullptr;        // rmax^3: right singular vectors per (slice, term)
  int* cn_kept = nullptr;        // kept terms a * r3 + c
  int* cn_count = nullptr;       // R* (device)
  double* cn_U = nullptr;        // 3 x n x cn_cap side matrices (row length cn_cap)
  double* cn_xi = nullptr;       // cn_cap weights
  int cn_cap = 0;                // capacity in terms
  int cn_rank = -1;              // R* of the current solve, -1 before rs_canonical
  // ALS refinement of the canonical-to-Tucker transform (allocated by the first rs_tucker_als call)
  double* als_Qp = nullptr;      // 3 x n x R_l x rmax: FP64 projections onto the current bases
  double* als_P = nullptr;       // n x als_kc: shifted long-range factor columns of one K chunk
  double* als_A = nullptr;       // als_kc x rmax^2: charge-weighted projected rows of one K chunk
  double* als_M = nullptr;       // n x rmax^2: the mode matrix M_{U_l}
  int* als_inv = nullptr;        // 3 x n: compacted index of each charged coordinate, -1 elsewhere
  int* als_start = nullptr;      // 3 x (n + 1): charged particles grouped by coordinate (CSR)
  int* als_items = nullptr;      // 3 x maxN
  int als_kc = 0;                // rows of one K chunk
  cudaEvent_t ev_part = nullptr, ev_bins = nullptr, ev_side = nullptr, ev_start = nullptr, ev_fac = nullptr;
  int n = 0, R = 0, R_l = 0, R_s = 0, L = 0;   // L = 2n - 1
  int ksub = 0;        // subspace width (multiple of KB)
  int rmax = 0;        // rank bound = leading dimension of Tucker factors
  int nbin = 0;        // bins per axis
  int maxN = 0;
  bool fp64 = true;
  double h = 0.0;
  int last_flags = 0;
  int last_N = 0;
  bool solved = false;
  std::string err;

  // device buffers
  double* pk64 = nullptr;   // R x L
  float*  pk32 = nullptr;   // R x L
  float*  pk32lo = nullptr; // R x L: p_k - pk32 (FP32 pairs of the factors)
  double* dpk64 = nullptr;  // R x L: derivatives of the factors in the centre offset
  float*  dpk32 = nullptr;  // R x L
  double* xyz = nullptr;    // maxN x 3 (copy of host input)
  double* Z = nullptr;      // maxN
  int*    j = nullptr;      // maxN x 3 grid indices
  int*    nz_idx = nullptr; // maxN, particles with nonzero charge (ascending)
  double* C = nullptr;      // 3 x n aggregated squared column weights
  int*    nzj = nullptr;    // 3 x n distinct coordinates with C > 0
  double* F = nullptr;      // L x L
  double* G = nullptr;      // 3 x n x n
  double* X = nullptr;      // 3 x n x ksub
  double* Q = nullptr;      // 3 x n x ksub
  double* Y = nullptr;      // 3 x n x ksub
  double* T = nullptr;      // 3 x ksub x ksub
  double* T2k = nullptr;    // 3 x ksub x ksub (scratch)
  double* W = nullptr;      // 3 x ksub x ksub
  double* W2 = nullptr;     // 3 x ksub x ksub
  int*    om_colptr = nullptr;  // ksub + 1: sparse embedding Omega (n x ksub) by column
  int*    om_row = nullptr;     // n * ZETA
  signed char* om_sgn = nullptr;
  double* part = nullptr;   // partial sums of the Gram-Schmidt kernel
  int*    order = nullptr;  // 3 x ksub eigenvalue order
  double* ev = nullptr;     // 3 x ksub sorted eigenvalues
  double* Z64 = nullptr;    // 3 x n x rmax Tucker bases
  float*  Z32 = nullptr;
  void*   Qp = nullptr;     // 3 x n x R_l x rmax projected factors (T)
  double* beta64 = nullptr; // rmax^3 FP64 accumulator
  void*   beta = nullptr;   // rmax^3 (T)
  void*   T1 = nullptr;     // rmax x rmax x n (T)
  void*   T2 = nullptr;     // rmax x n x n (T)
  int*    bin_count = nullptr;  // nbin^3 + 1
  int*    bin_start = nullptr;  // nbin^3 + 1
  int*    bin_items = nullptr;  // maxN (indices into nz list order)
  double* Epart = nullptr;      // energy partial sums
  int*    adims = nullptr;      // rmax: per-batch row counts of the mode-2 product
  int*    kdims = nullptr;      // rmax: per-batch inner sizes of the mode-2 product
  double* Fout = nullptr;       // maxN x 3 forces of the last solve
  // discrete gradient of the Tucker part (forces, rs_forces.cu)
  double* fd_w = nullptr;       // n x FD_WIDTH weights of the first-derivative rows (1/h included)
  int*    fd_s = nullptr;       // n: first grid index of each row's stencil
  double* dZ64 = nullptr;       // 3 x n x rmax: D_h applied to the Tucker bases
  float*  dZ32 = nullptr;
  void*   T1d = nullptr;        // 2 x n x rmax x rmax (T): beta x_3 V3 and beta x_3 (D_h V3), i3-major
  // RS interaction matrix products (rs_matvec.cu; allocated by the first call)
  int mv_M = 0, mv_logM = 0, mv_B = 0;   // circulant size, log2, fibre pairs per CTA
  void* mv_sym = nullptr;       // R x M symbols (T), divided by M
  void* mv_tw = nullptr;        // M/2 twiddles (complex T)
  void* mv_U = nullptr;         // n^3 (T) intermediates of the mode products
  void* mv_V = nullptr;
  void* mv_X = nullptr;         // n^3 (T) charge grid and product of the energy call
  void* mv_Y = nullptr;
  double* mv_E = nullptr;       // energy of the energy call (device)
  bool mv_symbols_ready = false;
  // tensor-core assembly of the FP32 output (rs_tc.cu), planned at create
  bool use_tc = false;
  int t2_ld = 0;                // i3 stride of T2 on the CUDA-core path
  int gamma_cap = 0;            // bound on the window half-width (host evaluation + 1)
  int tc_nch = 0, tc_Nc = 0;    // i1 chunks and chunk width (N of the MMAs)
  int tc_kpad = 0;              // K of the Tucker MMAs (rmax rounded to 16)
  int tc_ntiles = 0;            // output tiles of 128 consecutive grid points (i2, i3) of a plane
  int tc_na = 0, tc_ns = 0;     // stages of the T2 tiles and of the window operand pairs
  int tc_grid = 0;
  size_t tc_smem = 0;           // dynamic shared memory of the assembly kernel
  bool tc_staged = false;       // assembly epilogue through shared staging rows
  bool use_tc_core = false;     // tensor-core core contraction (FP32 bulk path)
  bool use_kr_core = false;     // ... in the Khatri-Rao form (operands formed once, bulk copies)
  void*   kmeta = nullptr;      // per K term of the core: Qp row offsets and charge (int4)
  void*   kr_buf = nullptr;     // Khatri-Rao operand window (FP16 hi / lo blocks)
  size_t  kr_bytes = 0;
  int     kr_passes = 0, kr_wstride = 0;
  double* pe = nullptr;         // per-particle pair energies (off-grid energy and forces)
  double* ewin = nullptr;       // window part of each charged particle's value (energy)
  long long wl_cap = 0;         // capacity of the window lists (entries)
  int*       wl_count = nullptr;   // ntiles + 1
  int*       wl_start = nullptr;   // ntiles + 1
  int4*      wl_rec = nullptr;     // wl_cap: (j1, j2, j3, float bits of z)
  int2*      wl_rng = nullptr;     // ntiles*nch: entries of each tile column per i1 chunk
  DevScalars* sc = nullptr;
  DevScalars* h_sc = nullptr;   // pinned host copy

  // stage profiling (CUDA events on c.stream, ring of PROF_RING solves)
  int launches = 0;             // kernels launched by the last solve
  bool profile = false;
  cudaEvent_t* prof_ev = nullptr;
  long long prof_count = 0;     // solves recorded since the last read
};

constexpr int NSTAGE = 9;
constexpr int PROF_RING = 512;

// Plain-data view of a context for kernels that evaluate the RS tensor at points.
struct DevView {
  int n, rmax, R, R_l, nbin;
  const DevScalars* sc;
  const int* bin_start;
  const int* bin_items;
  const int* j;
  const double* pk64;
  const double* Z;
  const int* nz_idx;
};

// Short-range windows at grid point (i1, i2, i3): adds this lane's share of
// sum_{nu in L(i)} z_nu U_nu(i) to v (Lemma 3.10 and Lemma 3.8, second term), FP64 factors; the
// lanes of a warp take the particle bins around the point in turn.
__device__ __forceinline__ void window_add(const DevView& c, int i1, int i2, int i3, int lane, double& v) {
  const int n = c.n;
  const int g = c.sc->gamma, L = 2 * n - 1, nb = c.nbin;
  const int b1a = max(0, i1 - g) / BIN, b1b = min(n - 1, i1 + g) / BIN;
  const int b2a = max(0, i2 - g) / BIN, b2b = min(n - 1, i2 + g) / BIN;
  const int b3a = max(0, i3 - g) / BIN, b3b = min(n - 1, i3 + g) / BIN;
  const int nb3 = b3b - b3a + 1, nb2 = b2b - b2a + 1;
  const int nbt = (b1b - b1a + 1) * nb2 * nb3;
  for (int t = lane; t < nbt; t += 32) {
    const int b3 = b3a + t % nb3, b2 = b2a + (t / nb3) % nb2, b1 = b1a + t / (nb3 * nb2);
    const int b = (b1 * nb + b2) * nb + b3;
    for (int it = c.bin_start[b]; it < c.bin_start[b + 1]; ++it) {
      const int q = c.bin_items[it];
      const int d1 = i1 - c.j[3 * q], d2 = i2 - c.j[3 * q + 1], d3 = i3 - c.j[3 * q + 2];
      if (abs(d1) > g || abs(d2) > g || abs(d3) > g) continue;
      double s = 0.0;
      for (int k = c.R_l; k < c.R; ++k) {
        const double* row = c.pk64 + (long long)k * L + n - 1;
        s += row[d1] * row[d2] * row[d3];
      }
      v += c.Z[q] * s;
    }
  }
}

// Gradient of the short-range windows at grid point (i1, i2, i3) (Defs. 3.4, 3.6 differentiated
// term by term): adds this lane's share of sum_{nu in L(i), nu != p} z_nu grad U_nu(i) to
// (g1, g2, g3), with the FP64 factor table and its derivatives in the centre offset (dpk64); the
// lanes of a warp take the particle bins around the point in turn.  The particle's own window
// (index p) is left out; its derivative at its own centre is zero in any case (p_k' is odd).
__device__ __forceinline__ void window_grad_add(const DevView& c, const double* __restrict__ dpk64, int i1,
                                                int i2, int i3, int p, int lane, double& g1, double& g2,
                                                double& g3) {
  const int n = c.n, L = 2 * n - 1;
  const int g = c.sc->gamma, nb = c.nbin;
  const int b1a = max(0, i1 - g) / BIN, b1b = min(n - 1, i1 + g) / BIN;
  const int b2a = max(0, i2 - g) / BIN, b2b = min(n - 1, i2 + g) / BIN;
  const int b3a = max(0, i3 - g) / BIN, b3b = min(n - 1, i3 + g) / BIN;
  const int nb3 = b3b - b3a + 1, nb2 = b2b - b2a + 1;
  const int nbt = (b1b - b1a + 1) * nb2 * nb3;
  for (int t = lane; t < nbt; t += 32) {
    const int b3 = b3a + t % nb3, b2 = b2a + (t / nb3) % nb2, b1 = b1a + t / (nb3 * nb2);
    const int b = (b1 * nb + b2) * nb + b3;
    for (int it = c.bin_start[b]; it < c.bin_start[b + 1]; ++it) {
      const int q = c.bin_items[it];
      if (q == p) continue;
      const int d1 = i1 - c.j[3 * q], d2 = i2 - c.j[3 * q + 1], d3 = i3 - c.j[3 * q + 2];
      if (abs(d1) > g || abs(d2) > g || abs(d3) > g) continue;
      double s1 = 0.0, s2 = 0.0, s3 = 0.0;
      for (int k = c.R_l; k < c.R; ++k) {
        const double* row = c.pk64 + (long long)k * L + n - 1;
        const double* drow = dpk64 + (long long)k * L + n - 1;
        const double f1 = row[d1], f2 = row[d2], f3 = row[d3];
        s1 += drow[d1] * f2 * f3;
        s2 += f1 * drow[d2] * f3;
        s3 += f1 * f2 * drow[d3];
      }
      const double zq = c.Z[q];
      g1 += zq * s1;
      g2 += zq * s2;
      g3 += zq * s3;
    }
  }
}

inline DevView make_view(const Ctx& c) {
  DevView v;
  v.n = c.n; v.rmax = c.rmax; v.R = c.R; v.R_l = c.R_l; v.nbin = c.nbin;
  v.sc = c.sc; v.bin_start = c.bin_start; v.bin_items = c.bin_items; v.j = c.j;
  v.pk64 = c.pk64; v.Z = c.Z; v.nz_idx = c.nz_idx;
  return v;
}

// ---------------------------------------------------------------- launchers
// Each launcher enqueues its kernels on c.stream and returns how many kernels it launched.
// setup (rs_setup.cu)
int launch_factors(Ctx& c);
int launch_prepare_particles(Ctx& c, int N, double min_sep, bool check_sep);   // snap, weights, nzj
int launch_compact_nz(Ctx& c, int N);   // charged particles, their count and sum |z|
int launch_gram_setup(Ctx& c);           // F matrix, Gram matrices cleared (configuration only)
int launch_gram(Ctx& c);                 // Gram matrices (after launch_gram_setup)
// eigen stage (rs_eigen.cu)
int launch_subspace(Ctx& c);
// Tucker stage (rs_tucker.cu)
int launch_projection_core(Ctx& c);
int launch_bins(Ctx& c);
int launch_recon_gemm(Ctx& c, void* out);
// tensor-core assembly (rs_tc.cu)
bool plan_assemble(Ctx& c);              // host: fills the tc_* fields, false if unsupported
size_t t2_tile_bytes(const Ctx& c);      // bytes of the tiled FP16 T2 (tensor-core path)
int launch_t2_tiles(Ctx& c);             // mode-2 product into tiled FP16 hi/lo operands
int launch_window_lists(Ctx& c);         // per-tile-column window lists
int launch_assemble(Ctx& c, float* out); // Tucker product + windows in one kernel
int launch_windows(Ctx& c, void* out);
int launch_energy(Ctx& c, int N);
int launch_forces(Ctx& c);              // long part from the untruncated pair kernel
// forces from the discrete gradient of the RS-Tucker tensor (rs_forces.cu)
constexpr int FD_ORDER = 8;             // order of the centred difference formula
constexpr int FD_WIDTH = FD_ORDER + 1;  // points per row
bool fd_table(int n, double h, double* w, int* start);   // host: the rows of D_h
int launch_forces_rs(Ctx& c);
// RS interaction matrix (rs_matvec.cu): Y = A X for n^3 tensors; the energy through it
int launch_matvec(Ctx& c, const void* X, void* Y, int which, bool offdiag, std::string& err);
int launch_energy_matvec(Ctx& c, std::string& err);
void free_matvec(Ctx& c);
cudaError_t set_attributes_matvec(int optin);

// Kernels launched with more than 48 KB of dynamic shared memory.  The limit is an attribute of
// the kernel (process-wide per device), so it is raised once per device to the opt-in maximum
// rather than to the size one context needs: contexts of different sizes then never lower it
// under one another, and no launch sets it concurrently with another thread's launch.
inline cudaError_t allow_max_dynamic_smem(const void* f, int optin) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, f);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
}
cudaError_t set_attributes_eigen(int optin);
cudaError_t set_attributes_tucker(int optin);
cudaError_t set_attributes_tc(int optin);
cudaError_t set_attributes_core(int optin);
int launch_core_tc(Ctx& c);
int launch_core_kr(Ctx& c);
size_t core_kr_plan(const Ctx& c, int& passes, int& wstride);
int launch_energy_t2(Ctx& c, double* part, int blocks);
int launch_energy_windows(Ctx& c);
int launch_canonical(Ctx& c, double eps, int r1, int r2, int r3, int P);
int launch_canonical_eval(Ctx& c, int M, const int* idx, double* out);
size_t canonical_svd_smem(int r);
size_t canonical_select_smem(int P);
cudaError_t set_attributes_canonical(int optin);
cudaError_t set_attributes_plain(int optin);
rs_status launch_plain(Ctx& c, int which, float* out);
rs_status launch_pair_energy_forces(Ctx& c, int N, const double* xyz, const double* Z, double* E, double* F);
int launch_eval_points(Ctx& c, int M, const int* idx, double* out);
// ALS refinement (rs_als.cu): FP64 projections of every mode onto its current basis
int launch_proj64(Ctx& c, double* Qp);
int als_refine(Ctx& c, int sweeps);      // kernels launched, or -1 with c.err set
void free_als(Ctx& c);

// generic batched GEMM on row-major matrices:
//   C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b]
// op(A) is M x K (A stored M x K with lda, or K x M when transA), op(B) is K x N.
// Fixed-point accumulation of the Tucker core.  Every partial sum of beta[a][b][c] (any subset
// of its terms z_K q1[K][a] q2[K][b] q3[K][c]) is bounded by B = R_l sum|z| qmax^3 (qmax the
// largest projection, recorded as a rounded float: factor 2 of margin), so with the scale 2^e,
// B 2^e < 2^61, the partial sums are 64-bit integers that add exactly: beta does not depend on
// the order of the atomic additions (2^-e is about 2^-61 B, far below FP64 rounding of beta).
__device__ __forceinline__ int beta_fx_shift(const DevScalars* sc, int R_l) {
  const double q = (double)__uint_as_float(sc->qmax_bits);
  const double B = 2.0 * R_l * sc->zabs_sum * q * q * q;
  if (!(B > 0.0) || !isfinite(B)) return 0;
  int E = 0;
  frexp(B, &E);                       // B < 2^E
  return max(-1000, min(1000, 61 - E));
}
// v 2^e as a 64-bit integer (pow2 = 2^e: the product is exact)
__device__ __forceinline__ unsigned long long beta_fx(double v, double pow2) {
  return (unsigned long long)__double2ll_rn(v * pow2);
}

// FP64 products with beta = 0 split K across CTAs deterministically through scr (partial tiles
// and per-tile arrival counters, zero between products); without scr they do not split.
template <typename T>
void gemm_batched(cudaStream_t s, bool transA, bool transB, int M, int N, int K,
                  T alpha, const T* A, int lda, long long sA,
                  const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC,
                  int batch, const int* dynM = nullptr, const int* dynN = nullptr,
                  const int* dynK = nullptr, const GemmScratch* scr = nullptr);

}  // namespace rs

#define RS_CUDA_OK(expr) (cudaSuccess == (expr))
