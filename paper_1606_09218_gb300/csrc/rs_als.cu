// ALS refinement of the canonical-to-Tucker transform (Sec. 6, steps (III)-(V)).
//
// Starting from the RHOSVD bases of the last solve (step (III)), every sweep updates the modes
// in the order l = 1, 2, 3 (step (IV)).  The long-range canonical tensor is projected onto the
// current bases of the other two modes l' < l'', which gives the n x (r_l' r_l'') matrix
//   M_{U_l}[i][(b,c)] = sum_{nu,k} z_nu p_k[i - j_l^nu] Qp_l'[j_l'^nu][k][b] Qp_l''[j_l''^nu][k][c]
// (xi_K w_nu^3 = z_nu).  Its dominant left singular vectors become the new basis of mode l: the
// eigenvectors of M M^T from the eigen stage of the solve, whose eps rule then gives the
// eps-truncated rank of M (the eps-truncation variant the text allows).  Step (V) reruns the
// projection and core of the solve with the final bases.
//
// Everything here is FP64.  The particles are grouped by their mode-l coordinate, so each
// charged coordinate j carries one row block A[(j,k)][(b,c)] = sum_{nu at j} z_nu q'[b] q''[c],
// and M = P A is one GEMM with P[i][(j,k)] = p_k[i - j] (K = charged coordinates x R_l, in
// chunks), followed by M M^T.
#include "rs_internal.cuh"

#include <algorithm>
#include <cstddef>

namespace rs {

// inv[l][nzj[l][q]] = q for the charged coordinates of mode l (inv is -1 elsewhere)
__global__ void als_inverse_kernel(const int* __restrict__ nzj, const DevScalars* sc, int n, int* inv) {
  const int l = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= sc->nzj_count[l]) return;
  const int jc = nzj[l * n + q];
  if (jc >= 0 && jc < n) inv[l * n + jc] = q;
}

// charged particles per compacted coordinate, counted at start[l][q + 1]
__global__ void als_count_kernel(const int* __restrict__ jidx, const int* __restrict__ nz_idx,
                                 const DevScalars* sc, int n, const int* __restrict__ inv, int* start) {
  const int l = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= sc->n_nz) return;
  const int q = inv[l * n + jidx[3 * nz_idx[m] + l]];
  if (q >= 0) atomicAdd(&start[l * (n + 1) + q + 1], 1);
}

// prefix sums of the counts (one thread per mode; at most n + 1 entries)
__global__ void als_scan_kernel(const DevScalars* sc, int n, int* start) {
  const int l = threadIdx.x;
  if (l >= 3) return;
  int* st = start + l * (n + 1);
  const int cnt = sc->nzj_count[l];
  for (int q = 1; q <= cnt; ++q) st[q] += st[q - 1];
}

// items[l][start[q] + rank] = particle, rank = its position among the charged particles of the
// same coordinate in ascending particle order (a fixed order: the sums over a coordinate's
// particles do not depend on the order of atomic operations)
__global__ void als_fill_kernel(const int* __restrict__ jidx, const int* __restrict__ nz_idx,
                                const DevScalars* sc, int n, int maxN, const int* __restrict__ inv,
                                const int* __restrict__ start, int* items) {
  const int l = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int nnz = sc->n_nz;
  if (m >= nnz) return;
  const int p = nz_idx[m];
  const int jl = jidx[3 * p + l];
  const int q = inv[l * n + jl];
  if (q < 0) return;
  int rank = 0;
  for (int m2 = 0; m2 < m; ++m2) rank += (jidx[3 * nz_idx[m2] + l] == jl);
  items[(long long)l * maxN + start[l * (n + 1) + q] + rank] = p;
}

// A[qq][(b,c)] for the K rows q = q0 + qq = (charged coordinate jq of mode l, long-range term k):
// sum over the particles at jq of z * Qp[o1][j_o1][k][b] * Qp[o2][j_o2][k][c]
__global__ void __launch_bounds__(256)
als_rows_kernel(const double* __restrict__ Qp, const int* __restrict__ jidx, const double* __restrict__ Z,
                const int* __restrict__ start, const int* __restrict__ items, int n, int R_l, int rmax,
                int maxN, int l, int o1, int o2, int r2, int Nd, int q0, double* A) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int qq = blockIdx.y;
  if (e >= Nd) return;
  const int q = q0 + qq, jq = q / R_l, k = q % R_l;
  const int b = e / r2, cc = e % r2;
  const int* st = start + l * (n + 1);
  const int* it = items + (long long)l * maxN;
  double s = 0.0;
  for (int t = st[jq]; t < st[jq + 1]; ++t) {
    const int p = it[t];
    const double* q1 = Qp + (((long long)o1 * n + jidx[3 * p + o1]) * R_l + k) * rmax;
    const double* q2 = Qp + (((long long)o2 * n + jidx[3 * p + o2]) * R_l + k) * rmax;
    s += Z[p] * q1[b] * q2[cc];
  }
  A[(long long)qq * Nd + e] = s;
}

// P[i][qq] = p_k[i - j] for the same K rows (j the charged coordinate of row q0 + qq)
__global__ void als_cols_kernel(const double* __restrict__ pk, const int* __restrict__ nzj, int n, int R_l,
                                int l, int q0, int kq, double* P) {
  const int qq = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (qq >= kq) return;
  const int q = q0 + qq, jq = q / R_l, k = q % R_l;
  const int jc = nzj[l * n + jq];
  P[(long long)i * kq + qq] = pk[(long long)k * (2 * n - 1) + (i - jc) + (n - 1)];
}

void free_als(Ctx& c) {
  for (void* p : {(void*)c.als_Qp, (void*)c.als_P, (void*)c.als_A, (void*)c.als_M, (void*)c.als_inv,
                  (void*)c.als_start, (void*)c.als_items})
    if (p) cudaFree(p);
  c.als_Qp = c.als_P = c.als_A = c.als_M = nullptr;
  c.als_inv = c.als_start = c.als_items = nullptr;
  c.als_kc = 0;
}

static bool als_alloc(Ctx& c) {
  const size_t n = (size_t)c.n, Rl = (size_t)c.R_l, rm = (size_t)c.rmax, r2 = rm * rm;
  // K chunk: A (chunk x rmax^2 doubles) within 128 MiB, whole factor rows, at most the grid's
  // limit of 65535 CTA rows
  size_t kc = ((size_t)1 << 24) / r2;
  kc = std::max(kc, Rl);
  kc = std::min(kc, n * Rl);
  kc = std::min<size_t>(kc, 65535);
  const size_t need[7] = {8 * 3 * n * Rl * rm, 8 * n * kc, 8 * kc * r2, 8 * n * r2, 4 * 3 * n,
                          4 * 3 * (n + 1), 4 * 3 * (size_t)std::max(c.maxN, 1)};
  void** dst[7] = {(void**)&c.als_Qp, (void**)&c.als_P, (void**)&c.als_A, (void**)&c.als_M,
                   (void**)&c.als_inv, (void**)&c.als_start, (void**)&c.als_items};
  for (int i = 0; i < 7; ++i) {
    if (cudaMalloc(dst[i], need[i]) != cudaSuccess) {
      cudaGetLastError();
      free_als(c);
      return false;
    }
  }
  c.als_kc = (int)kc;
  return true;
}

static bool read_scalars(Ctx& c) {
  cudaError_t e = cudaMemcpyAsync(c.h_sc, c.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c.err = std::string("tucker_als: ") + cudaGetErrorString(e);
    return false;
  }
  return true;
}

int als_refine(Ctx& c, int sweeps) {
  const int n = c.n, Rl = c.R_l, rm = c.rmax, maxN = std::max(c.maxN, 1);
  cudaStream_t s = c.stream;
  if (!c.als_Qp && !als_alloc(c)) {
    c.err = "tucker_als: device allocation failed";
    return -1;
  }
  if (!read_scalars(c)) return -1;
  const int nnz = c.h_sc->n_nz;
  if (nnz <= 0) return 0;                 // no charge: nothing to refine
  int k = 0;
  // charged particles grouped by coordinate, per mode
  cudaMemsetAsync(c.als_inv, 0xff, sizeof(int) * 3 * (size_t)n, s);
  cudaMemsetAsync(c.als_start, 0, sizeof(int) * 3 * (size_t)(n + 1), s);
  als_inverse_kernel<<<dim3((n + 255) / 256, 3), 256, 0, s>>>(c.nzj, c.sc, n, c.als_inv);
  als_count_kernel<<<dim3((nnz + 255) / 256, 3), 256, 0, s>>>(c.j, c.nz_idx, c.sc, n, c.als_inv, c.als_start);
  als_scan_kernel<<<1, 32, 0, s>>>(c.sc, n, c.als_start);
  als_fill_kernel<<<dim3((nnz + 255) / 256, 3), 256, 0, s>>>(c.j, c.nz_idx, c.sc, n, maxN, c.als_inv,
                                                           c.als_start, c.als_items);
  k += 4;
  // rows of uncharged coordinates are never written by the projection: keep them zero
  cudaMemsetAsync(c.als_Qp, 0, sizeof(double) * 3 * (size_t)n * Rl * rm, s);
  const size_t off_cnt = offsetof(DevScalars, bar_count), off_gen = offsetof(DevScalars, bar_gen);
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int l = 0; l < 3; ++l) {
      const int o1 = l == 0 ? 1 : 0, o2 = l == 2 ? 1 : 2;
      k += launch_proj64(c, c.als_Qp);    // projections onto the current bases
      if (!read_scalars(c)) return -1;    // current ranks
      const int r1 = c.h_sc->rank[o1], r2 = c.h_sc->rank[o2];
      const int cnt = c.h_sc->nzj_count[l];
      if (r1 <= 0 || r2 <= 0 || r1 > rm || r2 > rm || cnt <= 0 || cnt > n) continue;
      const int Nd = r1 * r2;
      const int Kd = cnt * Rl;
      // M = sum over K chunks of P A
      cudaMemsetAsync(c.als_M, 0, sizeof(double) * (size_t)n * Nd, s);
      for (int q0 = 0; q0 < Kd; q0 += c.als_kc) {
        const int kq = std::min(c.als_kc, Kd - q0);
        als_rows_kernel<<<dim3((Nd + 255) / 256, kq), 256, 0, s>>>(c.als_Qp, c.j, c.Z, c.als_start, c.als_items,
                                                                   n, Rl, rm, maxN, l, o1, o2, r2, Nd, q0,
                                                                   c.als_A);
        als_cols_kernel<<<dim3((kq + 255) / 256, n), 256, 0, s>>>(c.pk64, c.nzj, n, Rl, l, q0, kq, c.als_P);
        gemm_batched<double>(s, false, false, n, Nd, kq, 1.0, c.als_P, kq, 0, c.als_A, Nd, 0, 1.0, c.als_M, Nd, 0,
                             1);
        k += 3;
      }
      // G_l <- M M^T: the eigen stage then gives the dominant left singular vectors of M
      gemm_batched<double>(s, false, true, n, n, Nd, 1.0, c.als_M, Nd, 0, c.als_M, Nd, 0, 0.0,
                           c.G + (size_t)l * n * n, n, 0, 1, nullptr, nullptr, nullptr, &c.gscr);
      ++k;
      // the cooperative Gram-Schmidt kernel starts its mode barriers from generation zero
      cudaMemsetAsync((char*)c.sc + off_cnt, 0, sizeof(DevScalars::bar_count), s);
      cudaMemsetAsync((char*)c.sc + off_gen, 0, sizeof(DevScalars::bar_gen), s);
      // the other modes' Gram matrices are unchanged (the solve's, or the mode matrices of their
      // last update), so the eigen stage reproduces their current bases bit for bit
      k += launch_subspace(c);
    }
  }
  // step (V): projection and core with the final bases
  k += launch_projection_core(c);
  return k;
}

}  // namespace rs
