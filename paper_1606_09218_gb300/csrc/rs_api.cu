// C ABI of the RS library: context lifetime, workspace, and the per-solve pipeline
// (Sec. 2.2 factors -> Sec. 3.2 long-range Gram -> Sec. 6 RHOSVD -> Def. 3.9 RS-Tucker
// reconstruction with the windows of Def. 3.4 -> Sec. 4.2 energy).
#include "rs_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace rs;

struct rs_ctx {
  Ctx c;
};

namespace {

thread_local std::string g_create_err;

struct Sizes {
  int n, R, R_l, L, ks, rmax, nbin, maxN;
  bool fp64;
  size_t tsz;
  std::vector<std::pair<void**, size_t>> list;
};

bool derive(const rs_config& cfg, Ctx& c, std::string& err) {
  if (!(cfg.b > 0.0) || !std::isfinite(cfg.b)) { err = "b must be positive"; return false; }
  if (cfg.n < 5 || (cfg.n % 2) == 0) { err = "n must be odd and >= 5"; return false; }
  if (cfg.n > 2049) { err = "n above 2049 is not supported"; return false; }
  if (cfg.R < 2 || cfg.R > 64) { err = "R must be in [2, 64]"; return false; }
  if (cfg.R_s < 0 || cfg.R_s >= cfg.R || cfg.R_s > 16) { err = "need 0 <= R_s < R and R_s <= 16"; return false; }
  if (!(cfg.h_q > 0.0) || !std::isfinite(cfg.u0)) { err = "h_q must be positive and u0 finite"; return false; }
  if (!(cfg.eps > 0.0) || cfg.eps >= 1.0) { err = "eps must be in (0, 1)"; return false; }
  if (cfg.rank_cap < 0 || cfg.max_rank < 0) { err = "rank_cap and max_rank must be >= 0"; return false; }
  if (!(cfg.delta_rel >= 0.0)) { err = "delta_rel must be >= 0"; return false; }
  if (cfg.precision < RS_FP64 || cfg.precision > RS_FP32) { err = "unknown precision"; return false; }
  if (cfg.snap != 1) { err = "only snapped centres (snap = 1) are supported by rs_solve"; return false; }
  if (cfg.max_particles < 1) { err = "max_particles must be >= 1"; return false; }
  c.cfg = cfg;
  c.n = cfg.n;
  c.R = cfg.R;
  c.R_s = cfg.R_s;
  c.R_l = cfg.R - cfg.R_s;
  c.L = 2 * cfg.n - 1;
  c.h = 2.0 * cfg.b / (cfg.n - 1);
  c.fp64 = (cfg.precision == RS_FP64);
  int want = cfg.max_rank > 0 ? cfg.max_rank : 128;
  if (want > RMAX_LIMIT) want = RMAX_LIMIT;
  int ks = ((want + 16 + KB - 1) / KB) * KB;
  if (ks > KSUB_MAX) ks = KSUB_MAX;
  int nfloor = (cfg.n / KB) * KB;
  if (ks > nfloor) ks = nfloor;
  c.ksub = ks;
  c.rmax = want < ks ? want : ks;
  c.nbin = (cfg.n + BIN - 1) / BIN;
  c.maxN = cfg.max_particles;
  c.t2_ld = cfg.n;
  c.use_tc = plan_assemble(c);
  {
    // core contraction on the FP32 path: the Khatri-Rao tensor-core form where its operand
    // window takes at most a few passes over K; else the tensor-core form with operands built
    // per tile where the tolerance allows its FP32 accumulation (eps >= 1e-5), and the CUDA-core
    // two-sum contraction below that.  RS_CORE_PATH=cuda|tc|kr overrides.
    const char* env = std::getenv("RS_CORE_PATH");
    c.kr_bytes = c.fp64 ? 0 : core_kr_plan(c, c.kr_passes, c.kr_wstride);
    c.use_kr_core = c.kr_bytes > 0;
    c.use_tc_core = !c.fp64 && (c.use_kr_core || cfg.eps >= 1e-5);
    if (env && std::strcmp(env, "cuda") == 0) c.use_tc_core = c.use_kr_core = false;
    if (env && std::strcmp(env, "tc") == 0) {
      c.use_tc_core = !c.fp64;
      c.use_kr_core = false;
    }
    if (env && std::strcmp(env, "kr") == 0) c.use_tc_core = c.use_kr_core = c.kr_bytes > 0;
  }
  return true;
}

template <typename P>
void add(std::vector<std::pair<void**, size_t>>& v, P*& p, size_t bytes) {
  v.push_back({(void**)&p, bytes});
}

std::vector<std::pair<void**, size_t>> buffer_list(Ctx& c) {
  std::vector<std::pair<void**, size_t>> v;
  const size_t n = c.n, L = c.L, ks = c.ksub, rm = c.rmax, N = c.maxN, R = c.R, Rl = c.R_l;
  const size_t ts = c.fp64 ? 8 : 4;
  const size_t nbins = (size_t)c.nbin * c.nbin * c.nbin;
  add(v, c.pk64, 8 * R * L);
  add(v, c.pk32, 4 * R * L);
  add(v, c.pk32lo, 4 * R * L);
  add(v, c.dpk64, 8 * R * L);
  add(v, c.dpk32, 4 * R * L);
  add(v, c.xyz, 8 * 3 * N);
  add(v, c.Z, 8 * N);
  add(v, c.j, 4 * 3 * N);
  add(v, c.nz_idx, 4 * N);
  add(v, c.C, 8 * 3 * n);
  add(v, c.nzj, 4 * 3 * n);
  add(v, c.F, 8 * L * L);
  add(v, c.G, 8 * 3 * n * n);
  add(v, c.X, 8 * 3 * n * ks);
  add(v, c.Q, 8 * 3 * n * ks);
  add(v, c.Y, 8 * 3 * n * ks);
  add(v, c.T, 8 * 3 * ks * ks);
  add(v, c.T2k, 8 * 3 * ks * ks);
  add(v, c.W, 8 * 3 * ks * ks);
  add(v, c.W2, 8 * 3 * ks * ks);
  add(v, c.om_colptr, 4 * (ks + 1));
  add(v, c.om_row, 4 * n * ZETA);
  add(v, c.om_sgn, 1 * n * ZETA);
  // partials + reduced sums of the block Gram-Schmidt; before it, the rows' trace shares
  add(v, c.part, 8 * std::max<size_t>((size_t)(2 * 3 * NBC + 2 * 3) * (ks * KB + KB * KB), 6 * (size_t)n));
  add(v, c.order, 4 * 3 * ks);
  add(v, c.gscr.part, 8 * GEMM_SPLIT_SLOTS * 256);
  add(v, c.gscr.count, 4 * GEMM_SPLIT_SLOTS);
  add(v, c.ev, 8 * 3 * ks);
  add(v, c.Z64, 8 * 3 * n * rm);
  add(v, c.Z32, 4 * 3 * n * rm);
  add(v, c.Qp, ts * 3 * n * Rl * rm);
  if (c.use_tc_core) add(v, c.kmeta, 16 * (size_t)N * Rl);
  if (c.use_kr_core) add(v, c.kr_buf, c.kr_bytes);
  add(v, c.pe, 8 * (size_t)N);
  add(v, c.ewin, 8 * (size_t)N);
  add(v, c.beta64, 8 * rm * rm * rm);
  add(v, c.beta, ts * rm * rm * rm);
  add(v, c.T1, ts * rm * rm * n);
  add(v, c.T2, c.use_tc ? t2_tile_bytes(c) : ts * rm * n * (size_t)c.t2_ld);
  add(v, c.bin_count, 4 * (nbins + 1));
  add(v, c.bin_start, 4 * (nbins + 1));
  add(v, c.bin_items, 4 * N);
  add(v, c.Epart, 8 * ((N + 7) / 8 + 1));
  add(v, c.adims, 4 * rm);
  add(v, c.kdims, 4 * rm);
  add(v, c.Fout, 8 * 3 * N);
  add(v, c.fd_w, 8 * n * FD_WIDTH);
  add(v, c.fd_s, 4 * n);
  add(v, c.dZ64, 8 * 3 * n * rm);
  add(v, c.dZ32, 4 * 3 * n * rm);
  add(v, c.T1d, 2 * ts * rm * rm * n);
  add(v, c.sc, sizeof(DevScalars));
  if (c.use_tc) {
    const size_t nT = (size_t)c.tc_ntiles;
    add(v, c.wl_count, 4 * (nT + 1));
    add(v, c.wl_start, 4 * (nT + 1));
    add(v, c.wl_rec, 16 * (size_t)c.wl_cap);
    add(v, c.wl_rng, 8 * nT * c.tc_nch);
  }
  return v;
}

void free_profile(Ctx& c) {
  if (c.prof_ev) {
    for (int i = 0; i < PROF_RING * (NSTAGE + 1); ++i) cudaEventDestroy(c.prof_ev[i]);
    delete[] c.prof_ev;
    c.prof_ev = nullptr;
  }
  c.profile = false;
  c.prof_count = 0;
}

void free_canonical(Ctx& c) {
  for (void* p : {(void*)c.cn_sig, (void*)c.cn_X, (void*)c.cn_Y, (void*)c.cn_kept, (void*)c.cn_count, (void*)c.cn_U,
                  (void*)c.cn_xi})
    if (p) cudaFree(p);
  c.cn_sig = c.cn_X = c.cn_Y = c.cn_U = c.cn_xi = nullptr;
  c.cn_kept = c.cn_count = nullptr;
  c.cn_cap = 0;
  c.cn_rank = -1;
}

void free_all(Ctx& c) {
  free_profile(c);
  auto v = buffer_list(c);
  for (auto& e : v) {
    if (*e.first) cudaFree(*e.first);
    *e.first = nullptr;
  }
  if (c.h_sc) cudaFreeHost(c.h_sc);
  c.h_sc = nullptr;
  free_canonical(c);
  free_als(c);
  free_matvec(c);
  if (c.ev_part) cudaEventDestroy(c.ev_part);
  if (c.ev_bins) cudaEventDestroy(c.ev_bins);
  if (c.ev_side) cudaEventDestroy(c.ev_side);
  if (c.ev_start) cudaEventDestroy(c.ev_start);
  if (c.ev_fac) cudaEventDestroy(c.ev_fac);
  if (c.aux) cudaStreamDestroy(c.aux);
  c.ev_part = c.ev_bins = c.ev_side = c.ev_start = c.ev_fac = nullptr;
  c.aux = nullptr;
}

rs_status fail(Ctx& c, rs_status s, const std::string& msg) {
  c.err = msg;
  return s;
}

rs_status check_launch(Ctx& c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c.err = std::string(where) + ": " + cudaGetErrorString(e);
    return RS_ERR_CUDA;
  }
  return RS_OK;
}

rs_status sync_scalars(Ctx& c) {
  cudaError_t e = cudaMemcpyAsync(c.h_sc, c.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    c.err = std::string("synchronise: ") + cudaGetErrorString(e);
    return RS_ERR_CUDA;
  }
  return RS_OK;
}

rs_status status_of(const DevScalars& s) {
  if (s.flags & FLAG_TIMEOUT) return RS_ERR_TIMEOUT;
  if (s.flags & FLAG_OUTSIDE) return RS_ERR_OUTSIDE_BOX;
  if (s.flags & FLAG_WINDOWS) return RS_ERR_CAPACITY;
  if (s.flags & FLAG_SEPARATION) return RS_ERR_SEPARATION;
  if (s.flags & (FLAG_RANK_CAPPED | FLAG_CHOL)) return RS_RANK_CAPPED;
  return RS_OK;
}

}  // namespace

namespace rs {
// error text returned by rs_last_error(NULL) for calls without a context
void set_host_error(const std::string& msg) { g_create_err = msg; }
}  // namespace rs

extern "C" {

const char* rs_version(void) { return "rs-gb300 0.1 (sm_103a)"; }

size_t rs_workspace_bytes(const rs_config* cfg) {
  if (!cfg) return 0;
  Ctx c;
  std::string err;
  if (!derive(*cfg, c, err)) return 0;
  size_t tot = 0;
  for (auto& e : buffer_list(c)) tot += (e.second + 255) / 256 * 256;
  return tot;
}

namespace {

// raise the dynamic shared memory limit of the large-tile kernels once per device
bool ensure_kernel_attributes(std::string& err) {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    err = std::string("no CUDA device: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return true;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = set_attributes_eigen(optin);
  if (e == cudaSuccess) e = set_attributes_tucker(optin);
  if (e == cudaSuccess) e = set_attributes_tc(optin);
  if (e == cudaSuccess) e = set_attributes_core(optin);
  if (e == cudaSuccess) e = set_attributes_plain(optin);
  if (e == cudaSuccess) e = set_attributes_canonical(optin);
  if (e == cudaSuccess) e = set_attributes_matvec(optin);
  if (e != cudaSuccess) {
    err = std::string("kernel attributes: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return false;
  }
  done[dev] = true;
  return true;
}

}  // namespace

rs_status rs_create(const rs_config* cfg, void* stream, rs_ctx** out) {
  if (!cfg || !out) { g_create_err = "null argument"; return RS_ERR_INVALID_ARG; }
  *out = nullptr;
  rs_ctx* h = new (std::nothrow) rs_ctx();
  if (!h) { g_create_err = "host allocation failed"; return RS_ERR_OOM; }
  Ctx& c = h->c;
  std::string err;
  if (!derive(*cfg, c, err)) {
    g_create_err = err;
    delete h;
    return RS_ERR_INVALID_ARG;
  }
  c.stream = (cudaStream_t)stream;
  if (!ensure_kernel_attributes(err)) {
    g_create_err = err;
    delete h;
    return RS_ERR_CUDA;
  }
  // RS_DEBUG_POISON=1 fills every workspace buffer with 0xFF bytes (NaN / -1) so that a
  // read of memory the current solve did not write shows up in the results.
  const char* poison = std::getenv("RS_DEBUG_POISON");
  const bool do_poison = poison && poison[0] == '1';
  for (auto& e : buffer_list(c)) {
    cudaError_t st = cudaMalloc(e.first, e.second > 0 ? e.second : 1);
    if (st != cudaSuccess) {
      cudaGetLastError();
      g_create_err = std::string("device allocation failed: ") + cudaGetErrorString(st);
      free_all(c);
      delete h;
      return st == cudaErrorMemoryAllocation ? RS_ERR_OOM : RS_ERR_CUDA;
    }
    if (do_poison) cudaMemset(*e.first, 0xFF, e.second);
  }
  if (cudaMemset(c.gscr.count, 0, sizeof(unsigned) * GEMM_SPLIT_SLOTS) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "device memset failed";
    free_all(c);
    delete h;
    return RS_ERR_CUDA;
  }
  if (cudaMallocHost((void**)&c.h_sc, sizeof(DevScalars)) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "pinned host allocation failed";
    free_all(c);
    delete h;
    return RS_ERR_OOM;
  }
  std::memset(c.h_sc, 0, sizeof(DevScalars));
  if (cudaStreamCreateWithFlags(&c.aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.ev_part, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.ev_bins, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.ev_side, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.ev_start, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.ev_fac, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "stream or event creation failed";
    free_all(c);
    delete h;
    return RS_ERR_CUDA;
  }
  cudaMemsetAsync(c.sc, 0, sizeof(DevScalars), c.stream);
  // sparse sign embedding Omega (n x ksub, ZETA entries per row), stored by column
  {
    const int n = c.n, ks = c.ksub;
    std::vector<int> col(n * ZETA), cnt(ks + 1, 0), ptr(ks + 1, 0), row(n * ZETA);
    std::vector<signed char> sg(n * ZETA), sgc(n * ZETA);
    uint64_t state = 0x1606092181ull;
    auto next = [&]() {
      state += 0x9E3779B97F4A7C15ull;
      uint64_t x = state;
      x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
      x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
      return x ^ (x >> 31);
    };
    for (int i = 0; i < n * ZETA; ++i) {
      uint64_t r = next();
      col[i] = (int)(r % (uint64_t)ks);
      sg[i] = (r >> 63) ? 1 : -1;
      ++cnt[col[i]];
    }
    for (int m = 0; m < ks; ++m) ptr[m + 1] = ptr[m] + cnt[m];
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < n * ZETA; ++i) {
      int pos = fill[col[i]]++;
      row[pos] = i / ZETA;
      sgc[pos] = sg[i];
    }
    if (cudaMemcpy(c.om_colptr, ptr.data(), sizeof(int) * (ks + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.om_row, row.data(), sizeof(int) * n * ZETA, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.om_sgn, sgc.data(), n * ZETA, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      g_create_err = "upload of the range-finder embedding failed";
      free_all(c);
      delete h;
      return RS_ERR_CUDA;
    }
  }
  // rows of the first-derivative difference operator (forces)
  {
    std::vector<double> w((size_t)c.n * FD_WIDTH);
    std::vector<int> st(c.n);
    if (!fd_table(c.n, c.h, w.data(), st.data()) ||
        cudaMemcpy(c.fd_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.fd_s, st.data(), sizeof(int) * st.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      g_create_err = "upload of the difference operator failed";
      free_all(c);
      delete h;
      return RS_ERR_CUDA;
    }
  }
  *out = h;
  return RS_OK;
}

void rs_destroy(rs_ctx* h) {
  if (!h) return;
  cudaStreamSynchronize(h->c.stream);
  free_all(h->c);
  delete h;
}

rs_status rs_solve(rs_ctx* h, int N, const double* xyz, const double* Z, int flags,
                   double min_sep, void* potential_out) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  c.solved = false;
  c.cn_rank = -1;
  if (N < 0) return fail(c, RS_ERR_INVALID_ARG, "N must be >= 0");
  if (N > c.maxN) return fail(c, RS_ERR_CAPACITY, "N above max_particles of this context");
  if (N > 0 && (!xyz || !Z)) return fail(c, RS_ERR_INVALID_ARG, "null particle arrays");
  if ((flags & RS_POTENTIAL) && !potential_out)
    return fail(c, RS_ERR_INVALID_ARG, "RS_POTENTIAL needs potential_out");
  if ((flags & RS_POTENTIAL) && ((uintptr_t)potential_out & 15u))
    return fail(c, RS_ERR_INVALID_ARG, "potential_out must be 16-byte aligned");
  if ((flags & RS_VALIDATE_SEPARATION) && !(min_sep > 0.0))
    return fail(c, RS_ERR_INVALID_ARG, "RS_VALIDATE_SEPARATION needs min_sep > 0");
  if (flags & RS_INPUT_HOST) {
    // cheap host-side check before any device work
    for (long long i = 0; i < 3ll * N; ++i)
      if (!std::isfinite(xyz[i]) || std::fabs(xyz[i]) > c.cfg.b * (1.0 + 1e-12))
        return fail(c, RS_ERR_OUTSIDE_BOX, "particle outside [-b,b]^3 or non-finite coordinate");
    for (int i = 0; i < N; ++i)
      if (!std::isfinite(Z[i])) return fail(c, RS_ERR_OUTSIDE_BOX, "non-finite charge");
  }
  cudaStream_t s = c.stream;
  cudaEvent_t* ev = nullptr;
  if (c.profile) ev = c.prof_ev + (size_t)(c.prof_count % PROF_RING) * (NSTAGE + 1);
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], s); };
  int k = 0;
  cudaMemsetAsync(c.sc, 0, sizeof(DevScalars), s);
  if (N > 0) {
    cudaMemcpyKind kind = (flags & RS_INPUT_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaMemcpyAsync(c.xyz, xyz, sizeof(double) * 3 * N, kind, s);
    cudaMemcpyAsync(c.Z, Z, sizeof(double) * N, kind, s);
  }
  mark(0);
  // the configuration's factors, window width and F (a1, a2 and the F of a3), and the list of
  // charged particles, on the context's second stream beside the snapping and aggregation of the
  // particles: neither needs the other (so the "factors" stage of the profile is empty and the
  // "particles" stage covers both)
  cudaEventRecord(c.ev_start, s);
  cudaStreamWaitEvent(c.aux, c.ev_start, 0);
  c.stream = c.aux;
  k += launch_factors(c);                  // a1, a2: quadrature, factors, split, window width
  k += launch_gram_setup(c);               // a3: F = sum_k p_k p_k^T; Gram matrices cleared
  k += launch_compact_nz(c, N);            // the charged particles (needs only Z)
  cudaEventRecord(c.ev_fac, c.aux);
  c.stream = s;
  mark(1);
  k += launch_prepare_particles(c, N, min_sep, (flags & RS_VALIDATE_SEPARATION) != 0);
  cudaStreamWaitEvent(s, c.ev_fac, 0);
  mark(2);
  // particle bins and window lists need only the particles and gamma: on the context's second
  // stream, overlapped with the Gram and eigen stages (which leave most SMs idle)
  cudaEventRecord(c.ev_part, s);
  cudaStreamWaitEvent(c.aux, c.ev_part, 0);
  c.stream = c.aux;
  k += launch_bins(c);                     // window lists
  cudaEventRecord(c.ev_bins, c.aux);
  if ((flags & RS_ENERGY) && c.use_tc && !c.fp64)
    k += launch_energy_windows(c);         // a8, the neighbours' windows at every particle
  if ((flags & RS_FORCES) && (flags & RS_FORCES_PAIR)) k += launch_forces(c);   // a9, pair kernel
  c.stream = s;
  k += launch_gram(c);                     // a3, a4: Gram matrices of the long-range side matrices
  mark(3);
  k += launch_subspace(c);                 // a4: dominant subspaces, ranks
  mark(4);
  k += launch_projection_core(c);          // a5: projection and core
  mark(5);
  // (the energy's Tucker part stays on this stream after the assembly: beside it, its blocks
  // delay the persistent assembly CTAs more than they save)
  cudaEventRecord(c.ev_side, c.aux);
  cudaStreamWaitEvent(s, c.ev_bins, 0);    // window lists ready
  mark(6);
  rs_status st = check_launch(c, "solve");
  if (st != RS_OK) return st;
  if (flags & RS_POTENTIAL) k += launch_recon_gemm(c, potential_out);   // a7
  mark(7);
  if (flags & RS_POTENTIAL) k += launch_windows(c, potential_out);      // a6
  mark(8);
  cudaStreamWaitEvent(s, c.ev_side, 0);    // energy windows and forces (second stream) done
  if (flags & RS_ENERGY) k += launch_energy(c, N);                      // a8
  if ((flags & RS_FORCES) && !(flags & RS_FORCES_PAIR)) k += launch_forces_rs(c);   // a9
  mark(9);
  st = check_launch(c, "solve");
  if (st != RS_OK) return st;
  if (ev) ++c.prof_count;
  c.launches = k;
  c.last_flags = flags;
  c.last_N = N;
  c.solved = true;
  return RS_OK;
}

rs_status rs_energy(rs_ctx* h, double* E) {
  if (!h || !E) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.solved || !(c.last_flags & RS_ENERGY)) return fail(c, RS_ERR_NOT_READY, "no energy computed");
  // energy and flags only (the first 16 bytes of the device scalars)
  cudaError_t e = cudaMemcpyAsync(c.h_sc, c.sc, 16, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    c.err = std::string("synchronise: ") + cudaGetErrorString(e);
    return RS_ERR_CUDA;
  }
  *E = c.h_sc->energy;
  rs_status s2 = status_of(*c.h_sc);
  return s2 < 0 ? s2 : RS_OK;
}

rs_status rs_forces(rs_ctx* h, double* F, int to_host) {
  if (!h || !F) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.solved || !(c.last_flags & RS_FORCES)) return fail(c, RS_ERR_NOT_READY, "no forces computed");
  if (c.last_N > 0) {
    cudaError_t e = cudaMemcpyAsync(F, c.Fout, sizeof(double) * 3 * (size_t)c.last_N,
                                    to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c.stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c.err = std::string("forces copy: ") + cudaGetErrorString(e);
      return RS_ERR_CUDA;
    }
  }
  rs_status st = sync_scalars(c);
  if (st != RS_OK) return st;
  rs_status s2 = status_of(*c.h_sc);
  return s2 < 0 ? s2 : RS_OK;
}

rs_status rs_report(rs_ctx* h, rs_stats* out) {
  if (!h || !out) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.solved) return fail(c, RS_ERR_NOT_READY, "no solve");
  rs_status st = sync_scalars(c);
  if (st != RS_OK) return st;
  const DevScalars& s = *c.h_sc;
  std::memset(out, 0, sizeof(*out));
  out->N = c.last_N;
  out->N_nonzero = s.n_nz;
  double eb = 0.0;
  for (int l = 0; l < 3; ++l) {
    out->ranks[l] = s.rank[l];
    out->subspace[l] = s.k_eff[l];
    out->tail_rel[l] = s.tail_rel[l];
    eb += s.tail_rel[l];
  }
  out->eps_bound = std::sqrt(eb);
  out->gamma = s.gamma;
  out->P_R0 = s.P_R0;
  out->P_Rl0 = s.P_Rl0;
  out->energy = s.energy;
  out->status = status_of(s);
  out->kernel_launches = c.launches;
  return (rs_status)out->status;
}

rs_status rs_get_tucker(rs_ctx* h, int ranks[3], int* ld_V, int* ld_b, const void* V[3],
                        const void** beta) {
  if (!h || !ranks || !ld_V || !ld_b || !V || !beta) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.solved) return fail(c, RS_ERR_NOT_READY, "no solve");
  rs_status st = sync_scalars(c);
  if (st != RS_OK) return st;
  for (int l = 0; l < 3; ++l) {
    ranks[l] = c.h_sc->rank[l];
    V[l] = c.fp64 ? (const void*)(c.Z64 + (size_t)l * c.n * c.rmax)
                  : (const void*)(c.Z32 + (size_t)l * c.n * c.rmax);
  }
  *ld_V = c.rmax;
  *ld_b = c.rmax;
  *beta = c.beta;
  return RS_OK;
}

rs_status rs_get_windows(rs_ctx* h, int* n_s, int* R_s, int* N, const double** factors, int* ld_f,
                         const int** grid_idx, const double** charges) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!n_s || !R_s || !N || !factors || !ld_f || !grid_idx || !charges)
    return fail(c, RS_ERR_INVALID_ARG, "get_windows: null output");
  if (!c.solved) return fail(c, RS_ERR_NOT_READY, "no solve");
  rs_status st = sync_scalars(c);
  if (st != RS_OK) return st;
  const int g = c.h_sc->gamma;
  *n_s = 2 * g + 1;
  *R_s = c.R_s;
  *N = c.last_N;
  // the short-range rows of the factor table, from offset -gamma (the table holds the offsets
  // -(n-1)..(n-1), row length L)
  *factors = c.pk64 + (size_t)c.R_l * c.L + (size_t)(c.n - 1 - g);
  *ld_f = c.L;
  *grid_idx = c.j;
  *charges = c.Z;
  return RS_OK;
}

rs_status rs_eval_points(rs_ctx* h, int M, const int* idx, double* out) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.solved) return fail(c, RS_ERR_NOT_READY, "no solve");
  if (M < 0 || (M > 0 && (!idx || !out))) return fail(c, RS_ERR_INVALID_ARG, "bad point list");
  launch_eval_points(c, M, idx, out);
  return check_launch(c, "eval_points");
}

rs_status rs_canonical(rs_ctx* h, double eps, int* rank) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!rank || !(eps >= 0.0) || !std::isfinite(eps)) return fail(c, RS_ERR_INVALID_ARG, "rank pointer and eps >= 0");
  if (!c.solved) return fail(c, RS_ERR_NOT_READY, "no solve");
  int rk[3] = {0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(rk, c.sc->rank, sizeof(rk), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, RS_ERR_CUDA, std::string("canonical: ") + cudaGetErrorString(e));
  }
  const int r1 = rk[0], r2 = rk[1], r3 = rk[2];
  const int rm = r2 > r3 ? r2 : r3;
  const long long M = (long long)r1 * r3;
  if (rm > RS_CANONICAL_RMAX || M > RS_CANONICAL_TERMS)
    return fail(c, RS_ERR_CAPACITY, "canonical: Tucker ranks above the slice-SVD limits (112, 16384 terms)");
  const int cap = (int)(M > 0 ? M : 1);
  if (cap > c.cn_cap) {
    free_canonical(c);
    const size_t rmx = (size_t)c.rmax;
    const size_t need[7] = {8 * rmx * rmx, 8 * rmx * rmx * rmx, 8 * rmx * rmx * rmx, 4 * (size_t)cap, 4,
                            8 * 3 * (size_t)c.n * cap, 8 * (size_t)cap};
    void** dst[7] = {(void**)&c.cn_sig, (void**)&c.cn_X, (void**)&c.cn_Y, (void**)&c.cn_kept, (void**)&c.cn_count,
                     (void**)&c.cn_U, (void**)&c.cn_xi};
    for (int i = 0; i < 7; ++i) {
      if (cudaMalloc(dst[i], need[i]) != cudaSuccess) {
        cudaGetLastError();
        free_canonical(c);
        return fail(c, RS_ERR_OOM, "canonical: device allocation failed");
      }
    }
    c.cn_cap = cap;
  }
  if (M == 0) {
    cudaMemsetAsync(c.cn_count, 0, sizeof(int), c.stream);
  } else {
    int P = 1;
    while (P < M) P <<= 1;
    launch_canonical(c, eps, r1, r2, r3, P);
  }
  rs_status st = check_launch(c, "canonical");
  if (st != RS_OK) return st;
  int cnt = 0;
  e = cudaMemcpyAsync(&cnt, c.cn_count, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, RS_ERR_CUDA, std::string("canonical: ") + cudaGetErrorString(e));
  }
  c.cn_rank = cnt;
  *rank = cnt;
  return RS_OK;
}

rs_status rs_canonical_eval_points(rs_ctx* h, int M, const int* idx, double* out) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.solved || c.cn_rank < 0) return fail(c, RS_ERR_NOT_READY, "no canonical form of the current solve");
  if (M < 0 || (M > 0 && (!idx || !out))) return fail(c, RS_ERR_INVALID_ARG, "bad point list");
  launch_canonical_eval(c, M, idx, out);
  return check_launch(c, "canonical_eval_points");
}

rs_status rs_tucker_als(rs_ctx* h, int sweeps, int flags, void* potential_out) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (sweeps < 1 || sweeps > RS_ALS_MAX_SWEEPS) return fail(c, RS_ERR_INVALID_ARG, "tucker_als: sweeps in [1, 8]");
  if (flags & ~(RS_POTENTIAL | RS_ENERGY))
    return fail(c, RS_ERR_INVALID_ARG, "tucker_als: flags other than RS_POTENTIAL | RS_ENERGY");
  if ((flags & RS_POTENTIAL) && (!potential_out || ((uintptr_t)potential_out & 15u)))
    return fail(c, RS_ERR_INVALID_ARG, "tucker_als: RS_POTENTIAL needs a 16-byte aligned potential_out");
  if (!c.solved) return fail(c, RS_ERR_NOT_READY, "no solve");
  if ((flags & RS_ENERGY) && !(c.last_flags & RS_ENERGY))
    return fail(c, RS_ERR_NOT_READY, "tucker_als: RS_ENERGY needs a solve that computed the energy");
  rs_status st = sync_scalars(c);
  if (st != RS_OK) return st;
  const rs_status solved = status_of(*c.h_sc);
  if (solved < 0) return fail(c, solved, "tucker_als: the last solve failed");
  const int k = als_refine(c, sweeps);
  if (k < 0) {
    // an allocation failure happens before any change; a CUDA error may leave the Tucker part
    // half refined, so the results of the solve are withdrawn
    const bool oom = c.err.find("allocation") != std::string::npos;
    if (!oom) c.solved = false;
    return fail(c, oom ? RS_ERR_OOM : RS_ERR_CUDA, c.err);
  }
  c.cn_rank = -1;                          // the canonical form described the previous core
  int k2 = 0;
  if (flags & RS_POTENTIAL) {
    k2 += launch_recon_gemm(c, potential_out);
    k2 += launch_windows(c, potential_out);
  }
  if (flags & RS_ENERGY) k2 += launch_energy(c, c.last_N);
  // an energy not recomputed here belonged to the previous Tucker tensor
  c.last_flags = (c.last_flags & ~RS_ENERGY) | (flags & RS_ENERGY);
  c.launches = k + k2;
  st = check_launch(c, "tucker_als");
  if (st != RS_OK) return st;
  // device-side errors of the refinement (a bounded wait of the eigen stage that ran out)
  st = sync_scalars(c);
  if (st != RS_OK) return st;
  const rs_status dev = status_of(*c.h_sc);
  return dev < 0 ? dev : RS_OK;
}

rs_status rs_get_canonical(rs_ctx* h, int* rank, const double** xi, const double** U, int* ld) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!rank || !xi || !U || !ld) return fail(c, RS_ERR_INVALID_ARG, "null output");
  if (!c.solved || c.cn_rank < 0) return fail(c, RS_ERR_NOT_READY, "no canonical form of the current solve");
  *rank = c.cn_rank;
  *xi = c.cn_xi;
  *U = c.cn_U;
  *ld = c.cn_cap;
  return RS_OK;
}

rs_status rs_profile_enable(rs_ctx* h, int enable) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!enable) {
    cudaStreamSynchronize(c.stream);
    free_profile(c);
    return RS_OK;
  }
  if (c.profile) return RS_OK;
  c.prof_ev = new (std::nothrow) cudaEvent_t[PROF_RING * (NSTAGE + 1)];
  if (!c.prof_ev) return fail(c, RS_ERR_OOM, "profile events");
  for (int i = 0; i < PROF_RING * (NSTAGE + 1); ++i) {
    if (cudaEventCreate(&c.prof_ev[i]) != cudaSuccess) {
      cudaGetLastError();
      for (int q = 0; q < i; ++q) cudaEventDestroy(c.prof_ev[q]);
      delete[] c.prof_ev;
      c.prof_ev = nullptr;
      return fail(c, RS_ERR_CUDA, "cudaEventCreate failed");
    }
  }
  c.profile = true;
  c.prof_count = 0;
  return RS_OK;
}

rs_status rs_profile_read(rs_ctx* h, double* ms, int* nsolves) {
  if (!h || !ms || !nsolves) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.profile) return fail(c, RS_ERR_NOT_READY, "profiling is off");
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) {
    c.err = std::string("synchronise: ") + cudaGetErrorString(cudaGetLastError());
    return RS_ERR_CUDA;
  }
  for (int q = 0; q < NSTAGE; ++q) ms[q] = 0.0;
  long long cnt = c.prof_count < PROF_RING ? c.prof_count : PROF_RING;
  for (long long sidx = 0; sidx < cnt; ++sidx) {
    cudaEvent_t* ev = c.prof_ev + (size_t)sidx * (NSTAGE + 1);
    for (int q = 0; q < NSTAGE; ++q) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[q], ev[q + 1]) == cudaSuccess) ms[q] += t;
      else cudaGetLastError();
    }
  }
  *nsolves = (int)cnt;
  c.prof_count = 0;
  return RS_OK;
}

rs_status rs_debug_buffer(rs_ctx* h, const char* name, void** ptr, size_t* bytes) {
  if (!h || !name || !ptr || !bytes) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  cudaStreamSynchronize(c.stream);
  struct { const char* nm; void* p; } tab[] = {
      {"pk64", c.pk64}, {"F", c.F}, {"G", c.G}, {"C", c.C}, {"Q", c.Q}, {"X", c.X}, {"T", c.T},
      {"Z64", c.Z64}, {"beta64", c.beta64}, {"Qp", c.Qp}, {"T1", c.T1}, {"T2", c.T2},
      {"sc", c.sc}};
  for (auto& e : buffer_list(c)) {
    for (auto& t : tab) {
      if (std::strcmp(t.nm, name) == 0 && *e.first == t.p) {
        *ptr = t.p;
        *bytes = e.second;
        return RS_OK;
      }
    }
  }
  return fail(c, RS_ERR_INVALID_ARG, std::string("unknown buffer ") + name);
}

const char* rs_stage_name(int stage) {
  static const char* names[NSTAGE] = {"factors", "particles", "gram", "eigen", "core",
                                      "bins", "reconstruct", "windows", "energy"};
  return (stage >= 0 && stage < NSTAGE) ? names[stage] : nullptr;
}

static rs_status plain_entry(rs_ctx* h, float* out, int which) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.solved) return fail(c, RS_ERR_NOT_READY, "no solve");
  if (!out || ((uintptr_t)out & 3u)) return fail(c, RS_ERR_INVALID_ARG, "out must be a 4-byte aligned device buffer");
  const rs_status st = launch_plain(c, which, out);
  if (st != RS_OK) return fail(c, st, "grid too large for this plain-method kernel");
  return check_launch(c, which == 0 ? "plain_direct" : "plain_canonical");
}

rs_status rs_pair_energy_forces(rs_ctx* h, int N, const double* xyz, const double* Z, double* E, double* F) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (N < 0 || !E || (N > 0 && (!xyz || !Z))) return fail(c, RS_ERR_INVALID_ARG, "bad pair energy arguments");
  if (N > c.maxN) return fail(c, RS_ERR_CAPACITY, "N above max_particles of this context");
  const rs_status st = launch_pair_energy_forces(c, N, xyz, Z, E, F);
  if (st != RS_OK) return fail(c, st, "more quadrature terms than the pair kernel supports");
  return check_launch(c, "pair_energy_forces");
}

rs_status rs_matvec(rs_ctx* h, const void* X, void* Y, int flags) {
  if (!h) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!X || !Y || ((uintptr_t)X & 7u) || ((uintptr_t)Y & 7u) || X == Y)
    return fail(c, RS_ERR_INVALID_ARG, "matvec: X and Y must be distinct 8-byte aligned device buffers");
  if (flags & ~(RS_MATVEC_LONG | RS_MATVEC_SHORT | RS_MATVEC_OFFDIAG))
    return fail(c, RS_ERR_INVALID_ARG, "matvec: unknown flags");
  int which = flags & (RS_MATVEC_LONG | RS_MATVEC_SHORT);
  if (which == 0) which = RS_MATVEC_LONG | RS_MATVEC_SHORT;
  std::string err;
  const int k = launch_matvec(c, X, Y, which, (flags & RS_MATVEC_OFFDIAG) != 0, err);
  if (k < 0) return fail(c, RS_ERR_OOM, err);
  return check_launch(c, "matvec");
}

rs_status rs_energy_matvec(rs_ctx* h, double* E) {
  if (!h || !E) return RS_ERR_INVALID_ARG;
  Ctx& c = h->c;
  if (!c.solved) return fail(c, RS_ERR_NOT_READY, "no solve");
  std::string err;
  const int k = launch_energy_matvec(c, err);
  if (k < 0) return fail(c, RS_ERR_OOM, err);
  rs_status st = check_launch(c, "energy_matvec");
  if (st != RS_OK) return st;
  cudaError_t e = cudaMemcpyAsync(E, c.mv_E, sizeof(double), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, RS_ERR_CUDA, std::string("energy_matvec: ") + cudaGetErrorString(e));
  }
  st = sync_scalars(c);
  if (st != RS_OK) return st;
  const rs_status s2 = status_of(*c.h_sc);
  return s2 < 0 ? s2 : RS_OK;
}

rs_status rs_plain_direct(rs_ctx* h, float* out) { return plain_entry(h, out, 0); }
rs_status rs_plain_canonical(rs_ctx* h, float* out) { return plain_entry(h, out, 1); }

const char* rs_last_error(rs_ctx* h) {
  if (!h) return g_create_err.c_str();
  return h->c.err.c_str();
}

}  // extern "C"
