// C ABI of the GB300 generalized-Stokes solver: context lifetime, setup of
// the operators and multigrid hierarchy, and the entry points declared in
// include/stokes.h. No entry point lets a C++ exception escape: every error
// becomes a stokes_status plus a per-thread message.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace sk {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

void* Arena::raw(size_t bytes) {
  void* p = nullptr;
  SK_CUDA(cudaMalloc(&p, bytes));
  ptrs.push_back(p);
  return p;
}
void Arena::free_all() {
  for (void* p : ptrs) cudaFree(p);
  ptrs.clear();
}

void* VecPool::get(size_t elems, int esz) {
  uint64_t key = ((uint64_t)elems << 4) | (uint64_t)esz;
  auto it = free_.find(key);
  if (it != free_.end() && !it->second.empty()) {
    void* p = it->second.back();
    it->second.pop_back();
    return p;
  }
  return arena->raw(elems * esz + 16);
}
void VecPool::put(void* p, size_t elems, int esz) {
  uint64_t key = ((uint64_t)elems << 4) | (uint64_t)esz;
  free_[key].push_back(p);
}

// Dense SPD inverse via Cholesky (row-major, in place): A = L L^T, A^{-1} = L^{-T} L^{-1}.
static void spd_inverse(std::vector<double>& A, int m) {
  std::vector<double> L(A.size(), 0.0);
  for (int j = 0; j < m; ++j) {
    double s = A[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
    SK_REQUIRE(s > 0, STOKES_ERR_ARG, "coarse matrix is not positive definite");
    double d = std::sqrt(s);
    L[(size_t)j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double t = A[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      L[(size_t)i * m + j] = t / d;
    }
  }
  // W = L^{-1} (lower triangular)
  std::vector<double> W(A.size(), 0.0);
  for (int j = 0; j < m; ++j) {
    W[(size_t)j * m + j] = 1.0 / L[(size_t)j * m + j];
    for (int i = j + 1; i < m; ++i) {
      double t = 0;
      for (int k = j; k < i; ++k) t -= L[(size_t)i * m + k] * W[(size_t)k * m + j];
      W[(size_t)i * m + j] = t / L[(size_t)i * m + i];
    }
  }
  // A^{-1} = W^T W
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double t = 0;
      for (int k = std::max(i, j); k < m; ++k) t += W[(size_t)k * m + i] * W[(size_t)k * m + j];
      A[(size_t)i * m + j] = t;
    }
}

// Dense inverse of a coarsest-level matrix; a BSR3 matrix is expanded over the
// component-major unknowns (component r of node i at r * rows + i).
static void coarse_inverse(stokes_ctx& c, const Csr& M, double** out64) {
  const int rows = M.rows, bs = M.br;
  const int m = rows * bs;
  const size_t planes = (size_t)bs * bs;
  std::vector<int> rp(rows + 1), col(M.nnz);
  std::vector<double> v(planes * M.nnz);
  SK_CUDA(cudaMemcpyAsync(rp.data(), M.rowptr, sizeof(int) * (rows + 1), cudaMemcpyDeviceToHost, c.ex.s));
  SK_CUDA(cudaMemcpyAsync(col.data(), M.col, sizeof(int) * M.nnz, cudaMemcpyDeviceToHost, c.ex.s));
  SK_CUDA(cudaMemcpyAsync(v.data(), M.v64, sizeof(double) * planes * M.nnz, cudaMemcpyDeviceToHost, c.ex.s));
  SK_CUDA(cudaStreamSynchronize(c.ex.s));
  std::vector<double> A((size_t)m * m, 0.0);
  for (int i = 0; i < rows; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      for (int r = 0; r < bs; ++r)
        for (int q = 0; q < bs; ++q)
          A[(size_t)(r * rows + i) * m + (q * rows + col[k])] = v[(size_t)(r * bs + q) * M.nnz + k];
  spd_inverse(A, m);
  *out64 = c.arena.alloc<double>((size_t)m * m);
  SK_CUDA(cudaMemcpy(*out64, A.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice));
}

static float* f32_copy(stokes_ctx& c, const double* src, size_t n) {
  if (!src) return nullptr;
  float* d = c.arena.alloc<float>(n);
  to_f32(c.ex, src, d, n);
  return d;
}

// wall-clock milliseconds of the setup phases (stream synchronised at each mark)
struct PhaseClock {
  stokes_ctx& c;
  std::chrono::steady_clock::time_point t;
  explicit PhaseClock(stokes_ctx& cc) : c(cc), t(std::chrono::steady_clock::now()) {}
  void mark(int phase) {
    static const char* const names[STOKES_SETUP_PHASES] = {"setup: assembly", "setup: storage", "setup: coarse",
                                                           "setup: spectra",  "setup: copies",  "setup: tuning"};
    nvtxMarkA(names[phase]);  // the end of the phase on a profiler's timeline
    SK_CUDA(cudaStreamSynchronize(c.ex.s));
    const auto now = std::chrono::steady_clock::now();
    c.setup_ms[phase] += std::chrono::duration<double, std::milli>(now - t).count();
    t = now;
  }
};

void setup_context(stokes_ctx* cp, int n, const double* Xh) {
  NvtxRange range("stokes_setup");
  stokes_ctx& c = *cp;
  PhaseClock clock(c);
  c.n = n;
  c.ex.prof = &c.prof;
  c.prof.on = c.opt.profile != 0;
  c.prof.only = c.opt.profile >= 2 ? c.opt.profile - 2 : -1;
  c.pool.arena = &c.arena;
  c.mixed = c.opt.precision == STOKES_PRECISION_MIXED;
  c.sc.cap = 4096;
  c.sc.d = c.arena.alloc<double>(c.sc.cap);
  SK_CUDA(cudaMallocHost(&c.sc.h, sizeof(double) * c.sc.cap));
  c.ds.partial = c.arena.alloc<double>((size_t)kMaxDots * kDotBlocks);
  c.ds.counter = c.arena.alloc<unsigned>(1);
  SK_CUDA(cudaMemsetAsync(c.ds.counter, 0, sizeof(unsigned), c.ex.s));
  c.d_flag = c.arena.alloc<int>(1);
  c.ex.flag = c.d_flag;
  const unsigned evf = cudaEventDisableTiming | (c.opt.host_wait ? cudaEventBlockingSync : 0u);
  SK_CUDA(cudaEventCreateWithFlags(&c.ev_read, evf));
  SK_CUDA(cudaEventCreateWithFlags(&c.ev_sync, evf));

  // level sizes n -> ceil(n/2) -> ... down to at most 3 cubes per side (nested
  // Kuhn meshes when n is even, logical-coordinate transfers otherwise)
  std::vector<int> ns{n};
  while (ns.back() >= 4) ns.push_back((ns.back() + 1) / 2);
  std::vector<std::vector<double>> Xs(ns.size());
  Xs[0].assign(Xh, Xh + 3 * (size_t)(n + 1) * (n + 1) * (n + 1));
  for (size_t l = 1; l < ns.size(); ++l) {
    Xs[l].resize(3 * (size_t)(ns[l] + 1) * (ns[l] + 1) * (ns[l] + 1));
    subsample_vertices(ns[l - 1], ns[l], Xs[l - 1].data(), Xs[l].data());
  }
  for (double x : Xs[0]) SK_REQUIRE(std::isfinite(x), STOKES_ERR_ARG, "non-finite vertex coordinate");

  StencilTables* st = stencils_create(c.arena);
  c.lv.resize(ns.size());
  for (size_t l = 0; l < ns.size(); ++l) {
    Level& L = c.lv[l];
    L.n = ns[l];
    L.nvi = (2 * L.n - 1) * (2 * L.n - 1) * (2 * L.n - 1);
    L.np = (L.n + 1) * (L.n + 1) * (L.n + 1);
    L.X = c.arena.alloc<double>(Xs[l].size());
    SK_CUDA(cudaMemcpy(L.X, Xs[l].data(), sizeof(double) * Xs[l].size(), cudaMemcpyHostToDevice));
    Csr p2, p1, b, bt;
    build_pattern(c.ex, c.arena, st, PAT_P2P2, L.n, p2);
    build_pattern(c.ex, c.arena, st, PAT_P1P1, L.n, p1);
    const bool block_mg = c.opt.vel_prec != 3;
    AssemblyOut o;
    o.a3 = c.arena.alloc<double>(p2.nnz);
    o.kq = c.arena.alloc<double>(p1.nnz);
    if (block_mg) o.abs = c.arena.alloc<double>(9 * (size_t)p2.nnz);
    if (l == 0) {
      build_pattern(c.ex, c.arena, st, PAT_P1P2, L.n, b);
      build_pattern(c.ex, c.arena, st, PAT_P2P1, L.n, bt);
      if (!o.abs) o.abs = c.arena.alloc<double>(9 * (size_t)p2.nnz);
      o.mq = c.arena.alloc<double>(p1.nnz);
      o.lq = c.arena.alloc<double>(p1.nnz);
      o.b = c.arena.alloc<double>(3 * (size_t)b.nnz);
      o.bt = c.arena.alloc<double>(3 * (size_t)bt.nnz);
      o.lumped = c.arena.alloc<double>(L.nvi);
      if (c.opt.schur_prec == STOKES_SCHUR_PREC_MASS) o.mv = c.arena.alloc<double>(p2.nnz);
    }
    long long bad = assemble(c.ex, L.n, L.X, c.mu, c.dt, c.opt.eps_pressure, p2, p1, l == 0 ? &b : nullptr,
                             l == 0 ? &bt : nullptr, o, c.d_flag);
    SK_REQUIRE(bad == 0, STOKES_ERR_MESH,
               std::to_string(bad) + " inverted or degenerate tetrahedra on level " + std::to_string(l));
    L.A3 = p2;
    L.A3.v64 = o.a3;
    L.KQ = p1;
    L.KQ.v64 = o.kq;
    L.A3_dinv64 = c.arena.alloc<double>(L.A3.rows);
    L.KQ_dinv64 = c.arena.alloc<double>(L.KQ.rows);
    diag_inverse(c.ex, L.A3, L.A3_dinv64);
    diag_inverse(c.ex, L.KQ, L.KQ_dinv64);
    if (block_mg) {
      L.AV = p2;
      L.AV.br = L.AV.bc = 3;
      if (c.opt.vel_prec == 2) {
        L.AV.v64 = o.abs;  // A~_2 = A
      } else {
        L.AV.v64 = c.arena.alloc<double>(9 * (size_t)p2.nnz);
        combine_grad_div(c.ex, p2.nnz, o.abs, o.a3, c.gamma, L.AV.v64);
      }
      L.AV_dinv64 = c.arena.alloc<double>(3 * (size_t)L.AV.rows);
      diag_inverse(c.ex, L.AV, L.AV_dinv64);
    }
    if (l == 0) {
      c.A = p2;
      c.A.br = c.A.bc = 3;
      c.A.v64 = o.abs;
      c.MQ = p1;
      c.MQ.v64 = o.mq;
      c.LQ = p1;
      c.LQ.v64 = o.lq;
      c.B = b;
      c.B.br = 1;
      c.B.bc = 3;
      c.B.v64 = o.b;
      c.Bt = bt;
      c.Bt.br = 3;
      c.Bt.bc = 1;
      c.Bt.v64 = o.bt;
      c.lumped = o.lumped;
      if (o.mv) {
        c.MV = p2;
        c.MV.v64 = o.mv;
        c.MV_dinv64 = c.arena.alloc<double>(c.MV.rows);
        diag_inverse(c.ex, c.MV, c.MV_dinv64);
      }
    }
  }
  clock.mark(STOKES_SETUP_ASSEMBLY);
  for (size_t l = 0; l + 1 < c.lv.size(); ++l) {
    build_transfer_p2(c.ex, c.arena, c.lv[l].n, c.lv[l + 1].n, c.lv[l].P2, c.lv[l].R2);
    build_transfer_p1(c.ex, c.arena, c.lv[l].n, c.lv[l + 1].n, c.lv[l].P1, c.lv[l].R1);
  }
  if (c.opt.format != 1) {
    auto add = [&](Csr& m, int p2, int nn) {
      const int min_rows = c.opt.stencil_min_rows > 0 ? c.opt.stencil_min_rows : kStencilMinRows;
      const bool by_size = c.opt.format == 0 || c.opt.format == 3;
      if (by_size && m.rows < std::min(min_rows, kStencilMinRowsIL)) return;
      c.stencils.emplace_back(stencil_from_csr(c.ex, c.arena, st, p2, nn, m));
      m.st = c.stencils.back().get();
      m.st_min_single = by_size ? min_rows : 0;
    };
    for (Level& L : c.lv) {
      add(L.A3, 1, L.n);
      add(L.KQ, 0, L.n);
    }
    add(c.MQ, 0, n);
    add(c.LQ, 0, n);
    if (c.MV.v64) add(c.MV, 1, n);
  }
  if (c.opt.format != 1) {
    // the strain-form A also in symmetric stencil storage (half the values, no
    // indices): every product of A reads it (48^3, FP32, with the fused dot:
    // 171 us against 243 us for BSR3), and the double-float refinement
    // residual (324 against 421 us); format 3 keeps BSR3 for the products
    c.symA.reset(sym3_from_csr(c.ex, c.arena, st, n, c.A));
    c.A.sym = c.symA.get();
    c.A.sym_products = c.opt.format != 3;
  }
  // per-block partials of dot products fused into other kernels
  c.ds.fused_cap = std::max(std::max(kDotBlocks * kMaxBasis, bsr3_dot_grid(c.A)), c.symA ? sym3_grid(*c.symA) : 0);
  c.ds.fused_partial = c.arena.alloc<double>(c.ds.fused_cap);
  c.ds.fused_counter = c.arena.alloc<unsigned>(1);
  SK_CUDA(cudaMemsetAsync(c.ds.fused_counter, 0, sizeof(unsigned), c.ex.s));
  c.ds.k_cap = kdot_scratch(3 * (size_t)c.lv[0].nvi + c.lv[0].np, kMaxRhs);
  c.ds.k_partial = c.arena.alloc<double>((size_t)c.ds.k_cap);
  c.ds.k_counter = c.arena.alloc<unsigned>(kMaxRhs);
  SK_CUDA(cudaMemsetAsync(c.ds.k_counter, 0, sizeof(unsigned) * kMaxRhs, c.ex.s));
  clock.mark(STOKES_SETUP_STORAGE);
  Level& Lc = c.lv.back();
  coarse_inverse(c, Lc.A3, &Lc.A3_cinv64);
  coarse_inverse(c, Lc.KQ, &Lc.KQ_cinv64);
  if (Lc.AV.v64) coarse_inverse(c, Lc.AV, &Lc.AV_cinv64);
  clock.mark(STOKES_SETUP_COARSE);
  for (size_t l = 0; l + 1 < c.lv.size(); ++l) {
    c.lv[l].A3_lmax = estimate_lmax(c, c.lv[l].A3, c.lv[l].A3_dinv64, 15, 1000 + l);
    c.lv[l].KQ_lmax = estimate_lmax(c, c.lv[l].KQ, c.lv[l].KQ_dinv64, 15, 2000 + l);
    if (c.lv[l].AV.v64) c.lv[l].AV_lmax = estimate_lmax(c, c.lv[l].AV, c.lv[l].AV_dinv64, 15, 3000 + l);
  }
  clock.mark(STOKES_SETUP_SPECTRA);
  // fine-level auxiliaries
  const Level& L0 = c.lv[0];
  {
    std::vector<double> lum(L0.nvi);
    SK_CUDA(cudaMemcpy(lum.data(), c.lumped, sizeof(double) * L0.nvi, cudaMemcpyDeviceToHost));
    for (double& x : lum) x = 1.0 / x;
    c.lumped_inv64 = c.arena.alloc<double>(L0.nvi);
    SK_CUDA(cudaMemcpy(c.lumped_inv64, lum.data(), sizeof(double) * L0.nvi, cudaMemcpyHostToDevice));
  }
  c.MQ_dinv64 = c.arena.alloc<double>(L0.np);
  diag_inverse(c.ex, c.MQ, c.MQ_dinv64);
  {
    std::vector<double> ones(L0.np, 1.0);
    double* d1 = c.arena.alloc<double>(L0.np);
    SK_CUDA(cudaMemcpy(d1, ones.data(), sizeof(double) * L0.np, cudaMemcpyHostToDevice));
    c.MQ1 = c.arena.alloc<double>(L0.np);
    spmv_store<double>(c.ex, c.MQ, 1, d1, c.MQ1, -1);
    std::vector<double> h(L0.np);
    SK_CUDA(cudaMemcpyAsync(h.data(), c.MQ1, sizeof(double) * L0.np, cudaMemcpyDeviceToHost, c.ex.s));
    SK_CUDA(cudaStreamSynchronize(c.ex.s));
    c.MQ1_sum = 0;
    for (double x : h) c.MQ1_sum += x;
  }
  c.tet_vol = c.arena.alloc<double>(6 * (size_t)n * n * n);
  tet_volumes(c.ex, n, L0.X, c.tet_vol);
  c.U_last = c.arena.alloc<double>(3 * (size_t)L0.nvi);
  c.P_last = c.arena.alloc<double>(L0.np);
  if (c.mixed) {
    c.A.v32 = f32_copy(c, c.A.v64, 9 * (size_t)c.A.nnz);
    c.A.v32lo = c.arena.alloc<float>(9 * (size_t)c.A.nnz);
    to_f32_lo(c.ex, c.A.v64, c.A.v32, c.A.v32lo, 9 * (size_t)c.A.nnz);
    c.B.v32 = f32_copy(c, c.B.v64, 3 * (size_t)c.B.nnz);
    c.Bt.v32 = f32_copy(c, c.Bt.v64, 3 * (size_t)c.Bt.nnz);
    c.MQ.v32 = f32_copy(c, c.MQ.v64, c.MQ.nnz);
    c.LQ.v32 = f32_copy(c, c.LQ.v64, c.LQ.nnz);
    c.lumped_inv32 = f32_copy(c, c.lumped_inv64, L0.nvi);
    c.MQ_dinv32 = f32_copy(c, c.MQ_dinv64, L0.np);
    if (c.MV.v64) {
      c.MV.v32 = f32_copy(c, c.MV.v64, c.MV.nnz);
      c.MV_dinv32 = f32_copy(c, c.MV_dinv64, c.MV.rows);
    }
    for (Level& L : c.lv) {
      L.A3.v32 = f32_copy(c, L.A3.v64, L.A3.nnz);
      L.KQ.v32 = f32_copy(c, L.KQ.v64, L.KQ.nnz);
      L.A3_dinv32 = f32_copy(c, L.A3_dinv64, L.A3.rows);
      L.KQ_dinv32 = f32_copy(c, L.KQ_dinv64, L.KQ.rows);
      if (L.AV.v64) {
        L.AV.v32 = L.AV.v64 == c.A.v64 ? c.A.v32 : f32_copy(c, L.AV.v64, 9 * (size_t)L.AV.nnz);
        L.AV_dinv32 = f32_copy(c, L.AV_dinv64, 3 * (size_t)L.AV.rows);
      }
      for (Csr* t : {&L.P2, &L.R2, &L.P1, &L.R1})
        if (t->v64) t->v32 = f32_copy(c, t->v64, t->nnz);
    }
    for (auto& so : c.stencils) so->v32 = f32_copy(c, so->v64, so->total);
    if (c.symA) {
      c.symA->v32 = f32_copy(c, c.symA->v64, c.symA->total);
      c.symA->v32lo = c.arena.alloc<float>(c.symA->total);
      to_f32_lo(c.ex, c.symA->v64, c.symA->v32, c.symA->v32lo, c.symA->total);
    }
    Lc.A3_cinv32 = f32_copy(c, Lc.A3_cinv64, (size_t)Lc.A3.rows * Lc.A3.rows);
    Lc.KQ_cinv32 = f32_copy(c, Lc.KQ_cinv64, (size_t)Lc.KQ.rows * Lc.KQ.rows);
    if (Lc.AV_cinv64) Lc.AV_cinv32 = f32_copy(c, Lc.AV_cinv64, 9 * (size_t)Lc.AV.rows * Lc.AV.rows);
  }
  clock.mark(STOKES_SETUP_COPIES);
  // threads-per-row: tuned in the precision of the hot loop unless fixed by the caller
  auto tune = [&](Csr& m, int nr, int kind, int k = 1) {
    if (c.opt.spmv_group > 0) {
      int g = 1;
      while (g < c.opt.spmv_group && g < 32) g <<= 1;
      (k > 1 ? m.group4 : m.group) = g;
      return;
    }
    Csr probe = m;
    if (c.mixed && m.v32) probe.v64 = nullptr;
    autotune_group(c.ex, probe, nr, kind, k);
    m.group = probe.group;
    m.group4 = probe.group4;
  };
  tune(c.A, 3, 1);
  // threads per row of the symmetric A products: one (measured fastest inside
  // the solve at 48^3: 201 us against 232, 318, 508 us for 2, 4, 8) unless set
  if (c.A.sym) {
    c.symA->group = c.opt.spmv_group > 0 ? std::min(8, c.A.group) : 1;
    c.symA->batch = c.opt.sym_batch > 0 ? c.opt.sym_batch : 8;
  }
  tune(c.B, 1, 2);
  tune(c.Bt, 3, 3);
  tune(c.B, 1, 2, 4);  // four right-hand sides (stokes_solve_multi)
  tune(c.Bt, 3, 3, 4);
  tune(c.MQ, 1, 0);
  if (c.MV.v64) tune(c.MV, 3, 0);
  c.LQ.group = c.MQ.group;
  for (Level& L : c.lv) {
    tune(L.A3, 3, 0);
    tune(L.KQ, 1, 0);
    if (L.AV.v64) tune(L.AV, 3, 1);
    if (L.P2.rows) {
      tune(L.P2, 3, 0);
      tune(L.R2, 3, 0);
      tune(L.P1, 1, 0);
      tune(L.R1, 1, 0);
    }
  }
  clock.mark(STOKES_SETUP_TUNING);
}

}  // namespace sk

using namespace sk;

template <class F> static int guarded(F&& f) {
  try {
    f();
    return STOKES_OK;
  } catch (const sk::Error& e) {
    g_last_error = e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return STOKES_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return STOKES_ERR_CUDA;
  }
}

extern "C" {

void stokes_default_options(stokes_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->method = STOKES_METHOD_SCHUR;
  o->schur_prec = STOKES_SCHUR_PREC_LUMPED;
  o->precision = STOKES_PRECISION_FP64;
  o->vcycles = 2;
  o->cheb_degree = 2;
  o->mass_steps = 8;
  o->mass_steps_al = 24;
  o->restart = 30;
  o->block_lu = 1;
  o->m2_inner_cg = 0;
  o->inner_tol = 1e-10;
  o->schur_inner_tol = 1e-1;
  o->eps_pressure = 1.0;
  o->max_outer = 300;
  o->max_inner = 400;
  o->max_refine = 6;
  o->profile = 0;
  o->spmv_group = 0;
  o->schur_inner_iters = 2;
  o->pass_tol = 3e-2;
  o->format = 0;
  o->graphs = 1;
  o->vel_prec = 3;
  o->mass_steps_v = 8;
  o->coarse_kernel = 0;
  o->pass_schedule = 0;
  o->cheb_low = 0.1;
  o->cheb_high = 1.1;
  o->sym_batch = 0;
  o->stencil_min_rows = 0;
  o->host_wait = 0;
  o->vcycle_split = 1;
}

const char* stokes_status_string(int s) {
  switch (s) {
    case STOKES_OK: return "ok";
    case STOKES_ERR_ARG: return "invalid argument";
    case STOKES_ERR_OOM: return "out of device memory";
    case STOKES_ERR_CUDA: return "CUDA error";
    case STOKES_ERR_NOT_CONVERGED: return "not converged";
    case STOKES_ERR_BREAKDOWN: return "Krylov breakdown";
    case STOKES_ERR_NAN: return "non-finite value";
    case STOKES_ERR_TIMEOUT: return "device wait timed out";
    case STOKES_ERR_INCOMPATIBLE_RHS: return "incompatible pressure load (sum(g) != 0)";
    case STOKES_ERR_MESH: return "inverted or degenerate tetrahedron";
    default: return "unknown status";
  }
}

const char* stokes_last_error(void) { return g_last_error.c_str(); }

stokes_status stokes_setup(int n, const double* vertices, double mu, double dt, double gamma,
                           const stokes_options* opt, void* stream, stokes_ctx** out) {
  g_last_error.clear();
  if (!out || !vertices || n < 2 || !(mu > 0) || !(dt > 0) || !(gamma >= 0) || !std::isfinite(mu) ||
      !std::isfinite(dt) || !std::isfinite(gamma)) {
    g_last_error = "stokes_setup: need n >= 2, vertices, mu > 0, dt > 0, gamma >= 0 and out";
    return STOKES_ERR_ARG;
  }
  *out = nullptr;
  stokes_ctx* c = new (std::nothrow) stokes_ctx();
  if (!c) return STOKES_ERR_OOM;
  if (opt) c->opt = *opt; else stokes_default_options(&c->opt);
  if (c->opt.vcycles < 1 || c->opt.cheb_degree < 1 || c->opt.restart < 2 || !(c->opt.eps_pressure > 0) ||
      !(c->opt.inner_tol > 0) || !(c->opt.schur_inner_tol > 0) || c->opt.format < 0 || c->opt.format > 3 ||
      !(c->opt.pass_tol > 0 && c->opt.pass_tol < 1) || c->opt.vel_prec < 1 || c->opt.vel_prec > 3 ||
      c->opt.schur_prec < 0 || c->opt.schur_prec > 2 || c->opt.mass_steps_v < 1 ||
      c->opt.pass_schedule < 0 || c->opt.pass_schedule > 2 || !(c->opt.cheb_low > 0) ||
      !(c->opt.cheb_high > c->opt.cheb_low) || !std::isfinite(c->opt.cheb_high) ||
      !(c->opt.sym_batch == 0 || c->opt.sym_batch == 2 || c->opt.sym_batch == 4 || c->opt.sym_batch == 8) ||
      c->opt.host_wait < 0 || c->opt.host_wait > 1 || c->opt.vcycle_split < 0 || c->opt.vcycle_split > 2) {
    g_last_error = "stokes_setup: invalid options";
    delete c;
    return STOKES_ERR_ARG;
  }
  c->mu = mu;
  c->dt = dt;
  c->gamma = gamma;
  c->ex.s = (cudaStream_t)stream;
  int st = guarded([&]() { setup_context(c, n, vertices); });
  if (st != STOKES_OK) {
    std::string msg = g_last_error;
    stokes_destroy(c);
    g_last_error = msg;
    return (stokes_status)st;
  }
  *out = c;
  return STOKES_OK;
}

stokes_status stokes_solve(stokes_ctx* c, const double* f, const double* g, double tol, double* u, double* p,
                           stokes_info* info) {
  g_last_error.clear();
  if (!c || !f || !u || !p || !(tol > 0)) {
    g_last_error = "stokes_solve: null argument or tol <= 0";
    return STOKES_ERR_ARG;
  }
  int status = STOKES_OK;
  int st = guarded([&]() { status = solve_context(c, f, g, tol, u, p, info); });
  if (st != STOKES_OK) {
    if (info) info->status = st;
    return (stokes_status)st;
  }
  if (status != STOKES_OK) g_last_error = stokes_status_string(status);
  return (stokes_status)status;
}

stokes_status stokes_solve_multi(stokes_ctx* c, int k, const double* f, const double* g, double tol, double* u,
                                 double* p, stokes_info* info) {
  g_last_error.clear();
  if (!c || !f || !u || !p || !(tol > 0) || k < 1 || k > 4096) {
    g_last_error = "stokes_solve_multi: null argument, tol <= 0 or k outside [1, 4096]";
    return STOKES_ERR_ARG;
  }
  int status = STOKES_OK;
  int st = guarded([&]() { status = solve_multi_context(c, k, f, g, tol, u, p, info); });
  if (st != STOKES_OK) {
    if (info)
      for (int i = 0; i < k; ++i) info[i].status = st;
    return (stokes_status)st;
  }
  if (status != STOKES_OK) g_last_error = stokes_status_string(status);
  return (stokes_status)status;
}

stokes_status stokes_solve_host(stokes_ctx* c, const double* f, const double* g, double tol, double* u, double* p,
                                stokes_info* info) {
  g_last_error.clear();
  if (!c || !f || !u || !p || !(tol > 0)) {
    g_last_error = "stokes_solve_host: null argument or tol <= 0";
    return STOKES_ERR_ARG;
  }
  int status = STOKES_OK;
  int st = guarded([&]() {
    size_t N = (size_t)(2 * c->n + 1) * (2 * c->n + 1) * (2 * c->n + 1);
    size_t np = (size_t)c->lv[0].np;
    if (!c->f_dev) {
      c->f_dev = c->arena.alloc<double>(3 * N);
      c->u_dev = c->arena.alloc<double>(3 * N);
      c->g_dev = c->arena.alloc<double>(np);
      c->p_dev = c->arena.alloc<double>(np);
    }
    SK_CUDA(cudaMemcpyAsync(c->f_dev, f, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->ex.s));
    if (g) SK_CUDA(cudaMemcpyAsync(c->g_dev, g, sizeof(double) * np, cudaMemcpyHostToDevice, c->ex.s));
    status = solve_context(c, c->f_dev, g ? c->g_dev : nullptr, tol, c->u_dev, c->p_dev, info);
    SK_CUDA(cudaMemcpyAsync(u, c->u_dev, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->ex.s));
    SK_CUDA(cudaMemcpyAsync(p, c->p_dev, sizeof(double) * np, cudaMemcpyDeviceToHost, c->ex.s));
    SK_CUDA(cudaStreamSynchronize(c->ex.s));
  });
  if (st != STOKES_OK) return (stokes_status)st;
  if (status != STOKES_OK) g_last_error = stokes_status_string(status);
  return (stokes_status)status;
}

stokes_status stokes_adjoint(stokes_ctx* c, const double* dJdu, const double* dJdp, double tol, double* dJdf,
                             double* dJdg, double* dJdmu, stokes_info* info) {
  g_last_error.clear();
  if (!c || !dJdu || !dJdf || !(tol > 0)) {
    g_last_error = "stokes_adjoint: null argument or tol <= 0";
    return STOKES_ERR_ARG;
  }
  if (!c->have_solution) {
    g_last_error = "stokes_adjoint: call stokes_solve first";
    return STOKES_ERR_ARG;
  }
  int status = STOKES_OK;
  int st = guarded([&]() { status = adjoint_context(c, dJdu, dJdp, tol, dJdf, dJdg, dJdmu, info); });
  if (st != STOKES_OK) return (stokes_status)st;
  if (status != STOKES_OK) g_last_error = stokes_status_string(status);
  return (stokes_status)status;
}

stokes_status stokes_destroy(stokes_ctx* c) {
  if (!c) return STOKES_OK;
  cudaStreamSynchronize(c->ex.s);
  for (auto& row : c->cgraph)
    for (auto& g : row)
      if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& kv : c->vgraphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->prof.reset();
  if (c->ev_read) cudaEventDestroy(c->ev_read);
  if (c->ev_sync) cudaEventDestroy(c->ev_sync);
  if (c->sc.h) cudaFreeHost(c->sc.h);
  c->arena.free_all();
  delete c;
  return STOKES_OK;
}

stokes_status stokes_apply(stokes_ctx* c, int op, int level, const double* x, double* y) {
  g_last_error.clear();
  if (!c || !x || !y) {
    g_last_error = "stokes_apply: null argument";
    return STOKES_ERR_ARG;
  }
  return (stokes_status)guarded([&]() { apply_operator(c, op, level, x, y); });
}

static const Csr* matrix_of(stokes_ctx* c, int which, int level) {
  if (level < 0 || level >= (int)c->lv.size()) return nullptr;
  switch (which) {
    case STOKES_MAT_A: return level == 0 ? &c->A : nullptr;
    case STOKES_MAT_A3: return &c->lv[level].A3;
    case STOKES_MAT_B: return level == 0 ? &c->B : nullptr;
    case STOKES_MAT_BT: return level == 0 ? &c->Bt : nullptr;
    case STOKES_MAT_MQ: return level == 0 ? &c->MQ : nullptr;
    case STOKES_MAT_LQ: return level == 0 ? &c->LQ : nullptr;
    case STOKES_MAT_KQ: return &c->lv[level].KQ;
    case STOKES_MAT_AV: return c->lv[level].AV.v64 ? &c->lv[level].AV : nullptr;
    default: return nullptr;
  }
}

stokes_status stokes_matrix_shape(stokes_ctx* c, int which, int level, int64_t dims[5]) {
  g_last_error.clear();
  if (!c || !dims) return STOKES_ERR_ARG;
  if (which == STOKES_MAT_LUMPED) {
    if (level != 0) return STOKES_ERR_ARG;
    dims[0] = dims[1] = c->lv[0].nvi;
    dims[2] = c->lv[0].nvi;
    dims[3] = dims[4] = 1;
    return STOKES_OK;
  }
  const Csr* m = matrix_of(c, which, level);
  if (!m) {
    g_last_error = "stokes_matrix_shape: unknown matrix or level";
    return STOKES_ERR_ARG;
  }
  dims[0] = m->rows;
  dims[1] = m->cols;
  dims[2] = m->nnz;
  dims[3] = m->br;
  dims[4] = m->bc;
  return STOKES_OK;
}

stokes_status stokes_matrix_export(stokes_ctx* c, int which, int level, int32_t* rowptr, int32_t* colidx,
                                   double* vals) {
  g_last_error.clear();
  if (!c) return STOKES_ERR_ARG;
  return (stokes_status)guarded([&]() {
    if (which == STOKES_MAT_LUMPED) {
      SK_REQUIRE(level == 0 && vals, STOKES_ERR_ARG, "lumped mass: level 0 and vals required");
      SK_CUDA(cudaMemcpy(vals, c->lumped, sizeof(double) * c->lv[0].nvi, cudaMemcpyDeviceToHost));
      return;
    }
    const Csr* m = matrix_of(c, which, level);
    SK_REQUIRE(m && rowptr && colidx && vals, STOKES_ERR_ARG, "stokes_matrix_export: bad arguments");
    SK_CUDA(cudaStreamSynchronize(c->ex.s));
    SK_CUDA(cudaMemcpy(rowptr, m->rowptr, sizeof(int) * (m->rows + 1), cudaMemcpyDeviceToHost));
    SK_CUDA(cudaMemcpy(colidx, m->col, sizeof(int) * m->nnz, cudaMemcpyDeviceToHost));
    int bs = m->br * m->bc;
    std::vector<double> planes((size_t)bs * m->nnz);
    SK_CUDA(cudaMemcpy(planes.data(), m->v64, sizeof(double) * planes.size(), cudaMemcpyDeviceToHost));
    for (long long k = 0; k < m->nnz; ++k)
      for (int j = 0; j < bs; ++j) vals[(size_t)k * bs + j] = planes[(size_t)j * m->nnz + k];
  });
}

stokes_status stokes_sizes(stokes_ctx* c, int64_t sizes[6]) {
  if (!c || !sizes) return STOKES_ERR_ARG;
  int n = c->n;
  sizes[0] = n;
  sizes[1] = (int64_t)c->lv.size();
  sizes[2] = c->lv[0].nvi;
  sizes[3] = c->lv[0].np;
  sizes[4] = (int64_t)(2 * n + 1) * (2 * n + 1) * (2 * n + 1);
  sizes[5] = 3 * sizes[4] + sizes[3];
  return STOKES_OK;
}

stokes_status stokes_kernel_stats(stokes_ctx* c, int kernel, int64_t* launches, double* total_ms, double* bytes) {
  g_last_error.clear();
  if (!c || kernel < 0 || kernel >= STOKES_KERNEL_COUNT) return STOKES_ERR_ARG;
  return (stokes_status)guarded([&]() {
    SK_CUDA(cudaStreamSynchronize(c->ex.s));
    auto& r = c->prof.rec[kernel];
    double ms = 0;
    for (auto& p : r.ev) {
      float t = 0;
      SK_CUDA(cudaEventElapsedTime(&t, p.first, p.second));
      ms += t;
    }
    if (launches) *launches = r.launches;
    if (total_ms) *total_ms = ms;
    if (bytes) *bytes = r.bytes;
  });
}

stokes_status stokes_check_bounded_wait(stokes_ctx* c) {
  g_last_error.clear();
  if (!c) return STOKES_ERR_ARG;
  int status = STOKES_OK;
  int st = guarded([&]() {
    unsigned* bar = c->arena.alloc<unsigned>(1);
    SK_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->ex.s));
    bounded_wait_check(c->ex, bar);
    int flag = 0;
    SK_CUDA(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->ex.s));
    SK_CUDA(cudaStreamSynchronize(c->ex.s));
    SK_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->ex.s));
    SK_CUDA(cudaStreamSynchronize(c->ex.s));
    status = (flag & 4) ? STOKES_ERR_TIMEOUT : STOKES_OK;
  });
  if (st != STOKES_OK) return (stokes_status)st;
  if (status != STOKES_OK) g_last_error = "a device wait that nothing completes expired as designed";
  return (stokes_status)status;
}

stokes_status stokes_setup_phases(stokes_ctx* c, double ms[STOKES_SETUP_PHASES]) {
  if (!c || !ms) return STOKES_ERR_ARG;
  for (int k = 0; k < STOKES_SETUP_PHASES; ++k) ms[k] = c->setup_ms[k];
  return STOKES_OK;
}

stokes_status stokes_kernel_timing(stokes_ctx* c, int kernel, int64_t* timed_launches, double* timed_ms,
                                   double* timed_bytes) {
  g_last_error.clear();
  if (!c || kernel < 0 || kernel >= STOKES_KERNEL_COUNT) return STOKES_ERR_ARG;
  return (stokes_status)guarded([&]() {
    SK_CUDA(cudaStreamSynchronize(c->ex.s));
    auto& r = c->prof.rec[kernel];
    double ms = 0;
    for (auto& p : r.ev) {
      float t = 0;
      SK_CUDA(cudaEventElapsedTime(&t, p.first, p.second));
      ms += t;
    }
    if (timed_launches) *timed_launches = r.ev_launches;
    if (timed_ms) *timed_ms = ms;
    if (timed_bytes) *timed_bytes = r.ev_bytes;
  });
}

stokes_status stokes_kernel_stats_reset(stokes_ctx* c) {
  if (!c) return STOKES_ERR_ARG;
  return (stokes_status)guarded([&]() {
    SK_CUDA(cudaStreamSynchronize(c->ex.s));
    c->prof.reset();
  });
}

stokes_status stokes_profile_mode(stokes_ctx* c, int mode) {
  if (!c || mode < 0 || mode >= 2 + STOKES_KERNEL_COUNT) return STOKES_ERR_ARG;
  return (stokes_status)guarded([&]() {
    SK_CUDA(cudaStreamSynchronize(c->ex.s));
    c->opt.profile = mode;
    c->prof.on = mode != 0;
    c->prof.only = mode >= 2 ? mode - 2 : -1;
  });
}

}  // extern "C"
