// Allocation-free entry point: the Gram matrices of the long-range side matrices
// (the input of the eigen stage) computed with every scratch buffer in one file-scope
// device array instead of a context workspace.
//
// Some callers cannot call cudaMalloc: code that runs under a host application which has
// reserved all device memory up front and forbids further allocation, callers on a
// latency-critical path where an allocation (which may synchronise the device) is not
// acceptable, and plug-ins that may only use memory handed to them.  This entry point
// allocates nothing: the caller passes the particles and the output buffer, and the scratch
// lives in g_noalloc_scratch below.
#include "rs_internal.cuh"

#include <cmath>
#include <string>

namespace rs {
// kernels of the setup stage (rs_setup.cu), launched here on scratch inside the static array
__global__ void factors_kernel(double* pk64, float* pk32, float* pk32lo, double* dpk64, float* dpk32, int R,
                               int n, double h, double hq, double u0);
__global__ void scalars_kernel(const double* pk64, int R, int R_l, int n, double delta_rel,
                               DevScalars* sc);
__global__ void prepare_kernel(const double* xyz, const double* Z, int N, int n, double b,
                               double h, int* j, DevScalars* sc);
__global__ void aggregate_kernel(const double* xyz, const double* Z, int N, int n, double b, double h,
                                 double* C, const DevScalars* sc);
__global__ void compact_nzj_kernel(double* C, int n, int N, int* nzj, DevScalars* sc);
__global__ void fmatrix_kernel(const double* pk64, int R_l, int L, double* F);
__global__ void gram_kernel(const double* F, const double* C, const int* nzj,
                            const DevScalars* sc, int n, double* G);
void set_host_error(const std::string& msg);
}  // namespace rs

using namespace rs;

namespace {

// 16 MiB of scratch, held by every GPU that loads the library until the process exits.
constexpr size_t kNoAllocBytes = 16u << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" rs_status rs_gram_noalloc(const rs_config* cfg, int N, const double* xyz,
                                     const double* Z, double* G, void* stream) {
  if (!cfg || N < 0 || (N > 0 && (!xyz || !Z)) || !G) {
    set_host_error("rs_gram_noalloc: null or negative argument");
    return RS_ERR_INVALID_ARG;
  }
  const int n = cfg->n, R = cfg->R, R_s = cfg->R_s;
  if (!(cfg->b > 0.0) || n < 5 || (n % 2) == 0 || R < 2 || R > 64 || R_s < 0 || R_s >= R ||
      !(cfg->h_q > 0.0) || !std::isfinite(cfg->u0) || !(cfg->delta_rel >= 0.0)) {
    set_host_error("rs_gram_noalloc: invalid configuration");
    return RS_ERR_INVALID_ARG;
  }
  const int L = 2 * n - 1, R_l = R - R_s;
  // scratch layout: scalars | pk64 | C | nzj | F | j (the grid indices last: they grow with N)
  size_t off = 0;
  const size_t o_sc = off;   off = align256(off + sizeof(DevScalars));
  const size_t o_pk64 = off; off = align256(off + sizeof(double) * (size_t)R * L);
  const size_t o_C = off;    off = align256(off + sizeof(double) * 3 * (size_t)n);
  const size_t o_nzj = off;  off = align256(off + sizeof(int) * 3 * (size_t)n);
  const size_t o_F = off;    off = align256(off + sizeof(double) * (size_t)L * L);
  const size_t o_j = off;
  const size_t fixed = off;
  off = align256(off + sizeof(int) * 3 * (size_t)(N > 0 ? N : 1));
  if (off > kNoAllocBytes) {
    const long long nmax = fixed < kNoAllocBytes ? (long long)((kNoAllocBytes - fixed) / (3 * sizeof(int))) : 0;
    set_host_error("rs_gram_noalloc: problem needs " + std::to_string(off) +
                   " bytes of scratch, above the fixed 16 MiB (at n = " + std::to_string(n) + ", R = " +
                   std::to_string(R) + " up to N = " + std::to_string(nmax) + " centres fit)");
    return RS_ERR_CAPACITY;
  }
  // The device address of the array is looked up on every call (the lookup allocates
  // nothing): a cached address would be stale after the context of the device was reset.
  void* sym = nullptr;
  {
    cudaError_t e = cudaGetSymbolAddress(&sym, g_noalloc_scratch);
    if (e != cudaSuccess || !sym) {
      cudaGetLastError();
      set_host_error(std::string("rs_gram_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return RS_ERR_CUDA;
    }
  }
  unsigned char* base = (unsigned char*)sym;
  cudaStream_t s = (cudaStream_t)stream;
  DevScalars* sc = (DevScalars*)(base + o_sc);
  double* pk64 = (double*)(base + o_pk64);
  int* j = (int*)(base + o_j);
  double* C = (double*)(base + o_C);
  int* nzj = (int*)(base + o_nzj);
  double* F = (double*)(base + o_F);
  const double h = 2.0 * cfg->b / (n - 1);
  // the array keeps the previous call's contents: clear what is accumulated into
  cudaMemsetAsync(sc, 0, sizeof(DevScalars), s);
  cudaMemsetAsync(C, 0, sizeof(double) * 3 * (size_t)n, s);
  const int tot = R * L;
  factors_kernel<<<(tot + 255) / 256, 256, 0, s>>>(pk64, nullptr, nullptr, nullptr, nullptr, R, n, h, cfg->h_q,
                                                   cfg->u0);
  scalars_kernel<<<1, 256, 0, s>>>(pk64, R, R_l, n, cfg->delta_rel, sc);
  if (N > 0) {
    prepare_kernel<<<(N + 255) / 256, 256, 0, s>>>(xyz, Z, N, n, cfg->b, h, j, sc);
    aggregate_kernel<<<(N + 255) / 256, 256, 0, s>>>(xyz, Z, N, n, cfg->b, h, C, sc);
  }
  compact_nzj_kernel<<<3, 1024, 0, s>>>(C, n, N, nzj, sc);
  fmatrix_kernel<<<dim3((L + 255) / 256, L), 256, 0, s>>>(pk64, R_l, L, F);
  const int nt = (n + 31) / 32;
  gram_kernel<<<dim3(nt * (nt + 1) / 2, 3), 256, 0, s>>>(F, C, nzj, sc, n, G);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_host_error(std::string("rs_gram_noalloc: launch failed: ") + cudaGetErrorString(e));
    return RS_ERR_CUDA;
  }
  // the status word the particle kernels set: a centre outside the box or a non-finite input
  // leaves that particle out of the sums, so the call reports it instead of returning G
  unsigned flags = 0;
  e = cudaMemcpyAsync(&flags, &sc->flags, sizeof(flags), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_host_error(std::string("rs_gram_noalloc: ") + cudaGetErrorString(e));
    return RS_ERR_CUDA;
  }
  if (flags & FLAG_OUTSIDE) {
    set_host_error("rs_gram_noalloc: a centre outside [-b,b]^3 or a non-finite coordinate or charge");
    return RS_ERR_OUTSIDE_BOX;
  }
  return RS_OK;
}
