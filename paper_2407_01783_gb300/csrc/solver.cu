// Solver orchestration on one GPU stream: Chebyshev-Jacobi smoothing,
// geometric V-cycles, preconditioned CG, the Cahouet-Chabard Schur
// preconditioner, Method 1 (flexible CG on the pressure Schur complement,
// Sec. 2.3) and Method 2 (FGMRES on the coupled system with the block
// preconditioner of Eq. inexact_factorization_of_Alambda, Sec. 2.4), wrapped in
// defect correction on the full FP64 residual of Eq. Saddle_point_A_BT_B.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>
#include <type_traits>

#include "internal.h"

namespace sk {

void scalar_sub(const Exec& ex, double* out, const double* a, const double* b);


// sigma(D^{-1} M_Q) lies in [1/2, 5/2] for P1 on tetrahedra (element matrix
// D_K^{-1} M_K = (I + 1 1^T)/2 has eigenvalues 1/2 and 5/2; Wathen 1987).
constexpr double kMassLow = 0.5;
constexpr double kMassHigh = 2.5;
// sigma(D^{-1} M) for the P2 velocity mass: the element pencil (M_K, diag M_K)
// is the same for every affine tetrahedron (M_K = |K| M_ref), with extreme
// eigenvalues 1/4 and 4.34747 (rounded up); Wathen's element argument bounds
// the assembled (and Dirichlet-restricted) matrix by them
constexpr double kMassVLow = 0.25;
constexpr double kMassVHigh = 4.3475;

template <class T> static inline const T* pick(const double* a, const float* b);
template <> inline const double* pick<double>(const double* a, const float*) { return a; }
template <> inline const float* pick<float>(const double*, const float* b) { return b; }

// ---------------------------------------------------------------------------
// host reads of device scalars
// ---------------------------------------------------------------------------
// wait for all work issued on the context's stream (spinning or sleeping, as
// the event's flags say)
static void host_sync(stokes_ctx& c) {
  SK_CUDA(cudaEventRecord(c.ev_sync, c.ex.s));
  SK_CUDA(cudaEventSynchronize(c.ev_sync));
}
static double read_now(stokes_ctx& c, const double* d, int slot) {
  SK_CUDA(cudaMemcpyAsync(c.sc.h + slot, d, sizeof(double), cudaMemcpyDeviceToHost, c.ex.s));
  host_sync(c);
  return c.sc.h[slot];
}
static void read_issue(stokes_ctx& c, const double* d, int slot) {
  SK_CUDA(cudaMemcpyAsync(c.sc.h + slot, d, sizeof(double), cudaMemcpyDeviceToHost, c.ex.s));
  SK_CUDA(cudaEventRecord(c.ev_read, c.ex.s));
}
static double read_wait(stokes_ctx& c, int slot) {
  SK_CUDA(cudaEventSynchronize(c.ev_read));
  return c.sc.h[slot];
}

template <class T>
static void dot1(stokes_ctx& c, const T* x, const T* y, size_t n, double* out, int mode = kDotAuto) {
  const T* xs[1] = {x};
  const T* ys[1] = {y};
  dots<T>(c.ex, c.ds, 1, xs, ys, n, out, mode);
}
template <class T> static void copy(stokes_ctx& c, T* dst, const T* src, size_t n) {
  SK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, c.ex.s));
}
template <class T> static void zero(stokes_ctx& c, T* p, size_t n) {
  SK_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), c.ex.s));
}
// r <- r - mean(r) (Euclidean complement of the constants: pressure residuals
// live there because B^T 1 = 0)
template <class T> static void project_mean(stokes_ctx& c, T* r, size_t n, int mode = kDotExact) {
  int s = c.sc.take(1);
  dot1<T>(c, r, (const T*)nullptr, n, c.sc.d + s, mode);
  sub_mean<T>(c.ex, n, c.sc.d + s, (double)n, r);
  c.sc.give(1);
}

static size_t nvel(const stokes_ctx& c) { return 3 * (size_t)c.lv[0].nvi; }
static double nvi_of(const stokes_ctx& c) { return (double)c.lv[0].nvi; }
static size_t npres(const stokes_ctx& c) { return (size_t)c.lv[0].np; }

// ---------------------------------------------------------------------------
// Chebyshev semi-iteration for D^{-1} M on [lmin, lmax] (Saad, Alg. 12.1)
// ---------------------------------------------------------------------------
// layout: kLayoutIL (node-interleaved vectors of several right-hand sides,
// nr = 4 or 12) and / or kLayoutSplit (parity-split numbering, dinv in it too)
template <class T>
static void cheb_run(stokes_ctx& c, const Csr& M, int nr, const T* dinv, double lmin, double lmax, int steps,
                     const T* b, T* x, bool xzero, int kind, int layout = 0) {
  const bool il = layout & kLayoutIL;
  // a 3x3-block operator (M.br == 3) has one diagonal entry per component
  const bool block = M.br == 3;
  size_t len = (size_t)M.rows * (block ? 3 : nr);
  double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta, rho = 1.0 / sigma;
  Tmp<T> d(c.pool, len), xt(c.pool, len);
  // ping-pong between x and xt; from zero, start in xt when an odd number of
  // steps follows the first, so that the last step writes x (no copy)
  T* xa = x;
  T* xb = xt;
  if (xzero && (steps - 1) % 2 == 1) std::swap(xa, xb);
  auto step = [&](const T* xin, T* xout, double c1, double c2) {
    if (block) bsr3_cheb<T>(c.ex, M, b, xin, d, xout, dinv, c1, c2, kind);
    else spmv_cheb<T>(c.ex, M, nr, b, xin, d, xout, dinv, c1, c2, kind, layout);
  };
  if (xzero && !block && steps >= 2 && std::is_same<T, float>::value) {
    // the first two steps in one sweep (FP32: in FP64 the extra multiplies at
    // each gathered column load the scarce FP64 pipe more than the saved
    // streams relieve memory); the output buffer is picked so that the
    // remaining steps' ping-pong ends in x
    const double rn = 1.0 / (2.0 * sigma - rho);
    T* out = (steps - 2) % 2 == 0 ? x : (T*)xt;
    spmv_cheb_first<T>(c.ex, M, nr, b, d, out, dinv, 1.0 / theta, rn * rho, 2.0 * rn / delta, kind, layout);
    rho = rn;
    xa = out;
    xb = out == x ? (T*)xt : x;
    for (int k = 2; k < steps; ++k) {
      const double r2 = 1.0 / (2.0 * sigma - rho);
      step(xa, xb, r2 * rho, 2.0 * r2 / delta);
      std::swap(xa, xb);
      rho = r2;
    }
    if (xa != x) copy<T>(c, x, xa, len);
    return;
  }
  if (xzero) {
    if (il) cheb_first_il<T>(c.ex, len, nr, dinv, b, 1.0 / theta, d, xa);
    else cheb_first<T>(c.ex, len, block ? 1 : nr, dinv, b, 1.0 / theta, d, xa);
  } else {
    step(xa, xb, 0.0, 1.0 / theta);
    std::swap(xa, xb);
  }
  for (int k = 1; k < steps; ++k) {
    double rn = 1.0 / (2.0 * sigma - rho);
    step(xa, xb, rn * rho, 2.0 * rn / delta);
    std::swap(xa, xb);
    rho = rn;
  }
  if (xa != x) copy<T>(c, x, xa, len);
}

// M_Q^{-1} b by Chebyshev-Jacobi on the exact Wathen interval (K right-hand
// sides [K][np] in one sweep of M_Q)
template <class T> static void mass_inverse(stokes_ctx& c, const T* b, T* x, int steps, int K = 1) {
  const T* dinv = pick<T>(c.MQ_dinv64, c.MQ_dinv32);
  if (K == 4) {  // on node-interleaved copies (see vcycles_plain)
    const size_t rows = (size_t)c.MQ.rows;
    Tmp<T> bi(c.pool, rows * K), xi(c.pool, rows * K);
    to_interleaved<T>(c.ex, rows, K, b, bi);
    cheb_run<T>(c, c.MQ, K, dinv, kMassLow, kMassHigh, std::max(1, steps), bi, xi, true, STOKES_KERNEL_SPMV_P1,
                kLayoutIL);
    to_component_major<T>(c.ex, rows, K, xi, x);
    return;
  }
  cheb_run<T>(c, c.MQ, K, dinv, kMassLow, kMassHigh, std::max(1, steps), b, x, true, STOKES_KERNEL_SPMV_P1);
}

// ---------------------------------------------------------------------------
// geometric V-cycle; which = 0: A~_3 on 3 interleaved components, 1: eps M_Q + L_Q;
// K right-hand sides: 3K (resp. K) component-major components share every
// sweep of the level matrices
// ---------------------------------------------------------------------------
template <class T>
static void vcycle(stokes_ctx& c, int which, int l, const T* b, T* x, bool xzero, int K = 1, bool il = false,
                   bool split = false);

// Levels >= 1 are latency-bound (a few thousand rows per launch), so below
// level 0 the V-cycle is replayed from a CUDA graph. Graph launches are not
// timed per class: under per-class profiling of a class that the coarse
// levels launch, they run eagerly instead.
// Graph launches carry no per-launch events: graphs are off while every class
// is timed (profile 1); while one class is timed (profile 2 + k) they stay on
// and only that class's launches outside graphs are timed.
static bool coarse_graph_ok(const stokes_ctx& c, int which) {
  if (!c.opt.graphs || c.graphs_off || c.lv.size() < 2 || c.in_cycle_graph) return false;
  (void)which;
  return !c.prof.on || c.prof.only >= 0;
}

// swaps the context's vector pool with a graph's private one for a scope
struct PoolSwap {
  VecPool& a;
  VecPool& b;
  PoolSwap(VecPool& x, VecPool& y) : a(x), b(y) { std::swap(a.free_, b.free_); }
  ~PoolSwap() { std::swap(a.free_, b.free_); }
};

// ---------------------------------------------------------------------------
// The V-cycle below level 0 as an MgProgram (one cooperative kernel): the same
// steps, coefficients and buffer ping-pong as vcycle() and cheb_run() on the
// levels >= 1, recorded once with fixed buffers.
// ---------------------------------------------------------------------------
template <class T> static void mg_emit_cheb(stokes_ctx& c, MgProgram& P, const Csr& M, int nr, const T* dinv,
                                           double lmin, double lmax, int steps, const T* b, T* x, bool xzero) {
  const size_t len = (size_t)M.rows * nr;
  T* d = c.arena.alloc<T>(len);
  T* xt = c.arena.alloc<T>(len);
  double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta, rho = 1.0 / sigma;
  T* xa = x;
  T* xb = xt;
  if (xzero && (steps - 1) % 2 == 1) std::swap(xa, xb);
  auto csr_step = [&](const T* xin, T* xout, double c1, double c2) {
    MgOp o;
    o.kind = 4;
    o.nr = nr;
    o.rows = M.rows;
    o.m = M.cols;
    o.rp = M.rowptr;
    o.col = M.col;
    o.val = M.template v<T>();
    o.b = b;
    o.xin = xin;
    o.d = d;
    o.y = xout;
    o.dinv = dinv;
    o.c1 = c1;
    o.c2 = c2;
    P.add(o);
    P.bytes += M.bytes(sizeof(T)) + (double)sizeof(T) * len * 6 + (double)sizeof(T) * M.rows;
  };
  if (xzero) {
    MgOp o;
    o.kind = 0;
    o.nr = nr;
    o.rows = M.rows;
    o.b = b;
    o.d = d;
    o.y = xa;
    o.dinv = dinv;
    o.c1 = 1.0 / theta;
    P.add(o);
    P.bytes += (double)sizeof(T) * (3.0 * len + M.rows);
  } else {
    csr_step(xa, xb, 0.0, 1.0 / theta);
    std::swap(xa, xb);
  }
  for (int k = 1; k < steps; ++k) {
    double rn = 1.0 / (2.0 * sigma - rho);
    csr_step(xa, xb, rn * rho, 2.0 * rn / delta);
    std::swap(xa, xb);
    rho = rn;
  }
  SK_REQUIRE(xa == x, STOKES_ERR_ARG, "multigrid program: odd post-smoothing step count");
}

template <class T> static void mg_emit_csr(stokes_ctx& c, MgProgram& P, int kind, const Csr& M, int nr,
                                          const T* b, const T* x, T* y) {
  MgOp o;
  o.kind = kind;
  o.nr = nr;
  o.rows = M.rows;
  o.m = M.cols;
  o.rp = M.rowptr;
  o.col = M.col;
  o.val = M.template v<T>();
  o.b = b;
  o.xin = x;
  o.y = y;
  P.add(o);
  P.bytes += M.bytes(sizeof(T)) + (double)sizeof(T) * nr * ((double)M.cols + M.rows * (kind == 1 ? 1.0 : 2.0));
  (void)c;
}

template <class T> static void mg_emit_vcycle(stokes_ctx& c, MgProgram& P, int which, int l, const T* b, T* x) {
  Level& L = c.lv[l];
  const int nr = which == 1 ? 1 : 3;
  const Csr& M = which == 1 ? L.KQ : L.A3;
  if (l + 1 == (int)c.lv.size()) {
    MgOp o;
    o.kind = 5;
    o.nr = nr;
    o.m = M.rows;
    o.val = which ? pick<T>(L.KQ_cinv64, L.KQ_cinv32) : pick<T>(L.A3_cinv64, L.A3_cinv32);
    o.b = b;
    o.y = x;
    P.add(o);
    P.bytes += (double)sizeof(T) * ((double)M.rows * M.rows + 2.0 * M.rows * nr);
    return;
  }
  const T* dinv = which == 1 ? pick<T>(L.KQ_dinv64, L.KQ_dinv32) : pick<T>(L.A3_dinv64, L.A3_dinv32);
  const double lhat = which == 1 ? L.KQ_lmax : L.A3_lmax;
  const int deg = std::max(1, c.opt.cheb_degree);
  mg_emit_cheb<T>(c, P, M, nr, dinv, c.opt.cheb_low * lhat, c.opt.cheb_high * lhat, deg, b, x, true);
  const size_t len = (size_t)M.rows * nr;
  Level& Lc = c.lv[l + 1];
  const size_t lenc = (size_t)(which == 1 ? Lc.KQ.rows : Lc.A3.rows) * nr;
  T* r = c.arena.alloc<T>(len);
  T* bc = c.arena.alloc<T>(lenc);
  T* xc = c.arena.alloc<T>(lenc);
  mg_emit_csr<T>(c, P, 3, M, nr, b, x, r);                                  // r = b - M x
  mg_emit_csr<T>(c, P, 1, which == 1 ? L.R1 : L.R2, nr, nullptr, r, bc);   // bc = R r
  mg_emit_vcycle<T>(c, P, which, l + 1, bc, xc);
  mg_emit_csr<T>(c, P, 2, which == 1 ? L.P1 : L.P2, nr, nullptr, xc, x);   // x += P xc
  mg_emit_cheb<T>(c, P, M, nr, dinv, c.opt.cheb_low * lhat, c.opt.cheb_high * lhat, deg, b, x, false);
}

// The program for the levels >= 1 of V-cycle kind `which` (0: A~_3, 1: eps
// M_Q + L_Q), built on first use; its input b and output x are fixed buffers.
template <class T> static MgProgram* mg_program(stokes_ctx& c, int which) {
  auto& slot = c.mgprog[which][std::is_same<T, float>::value ? 1 : 0];
  if (!slot) {
    SK_REQUIRE(c.lv.size() >= 2, STOKES_ERR_ARG, "multigrid program needs two levels");
    auto P = std::make_unique<MgProgram>();
    const int nr = which == 1 ? 1 : 3;
    const size_t len1 = (size_t)(which == 1 ? c.lv[1].KQ.rows : c.lv[1].A3.rows) * nr;
    P->b = c.arena.alloc<T>(len1);
    P->x = c.arena.alloc<T>(len1);
    mg_emit_vcycle<T>(c, *P, which, 1, (const T*)P->b, (T*)P->x);
    P->finalize(c.arena, std::is_same<T, float>::value);
    slot = std::move(P);
  }
  return slot.get();
}

// the cooperative kernel serves V-cycles of A~_3 and eps M_Q + L_Q when the
// hierarchy has a level below the first coarse one and the cycle uses
// Chebyshev smoothing with an even number of steps after the first (so the
// smoothed iterate ends in its own buffer)
static bool coarse_kernel_ok(const stokes_ctx& c, int which) {
  return c.opt.coarse_kernel && which != 2 && c.lv.size() >= 3 && std::max(1, c.opt.cheb_degree) % 2 == 0;
}

// x_1 = V-cycle below level 0 applied to b_1 (G.b -> G.x)
template <class T> static void coarse_run(stokes_ctx& c, int which, stokes_ctx::CoarseGraph& G) {
  PoolSwap swap(c.pool, G.pool);
  if (G.state == 0) {  // eager: fills the private pool with every temporary
    vcycle<T>(c, which, 1, (const T*)G.b, (T*)G.x, true);
    G.state = 1;
    return;
  }
  if (G.state == 1) {
    if (!c.cap_stream) SK_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    G.counts = Prof::Counts{};
    const cudaStream_t launch = c.ex.s;
    cudaGraph_t g = nullptr;
    SK_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    c.prof.capture = &G.counts;
    c.ex.s = c.cap_stream;
    try {
      vcycle<T>(c, which, 1, (const T*)G.b, (T*)G.x, true);
    } catch (...) {
      c.ex.s = launch;
      c.prof.capture = nullptr;
      cudaStreamEndCapture(c.cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    c.ex.s = launch;
    c.prof.capture = nullptr;
    SK_CUDA(cudaStreamEndCapture(c.cap_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    SK_CUDA(e);
    G.state = 2;
  }
  SK_CUDA(cudaGraphLaunch(G.exec, c.ex.s));
  if (c.prof.on)
    for (int k = 0; k < STOKES_KERNEL_COUNT; ++k) {
      c.prof.rec[k].launches += G.counts.launches[k];
      c.prof.rec[k].bytes += G.counts.bytes[k];
    }
}

// level operator of V-cycle kind `which`
static const Csr& level_op(const Level& L, int which) { return which == 1 ? L.KQ : (which == 2 ? L.AV : L.A3); }

// residual r = b - M x of a level operator (scalar with nr components or 3x3 blocks)
template <class T>
static void level_resid(stokes_ctx& c, const Csr& M, int nr, const T* b, const T* x, T* r, int kind, int layout = 0) {
  if (M.br == 3) bsr3_apply<T>(c.ex, M, x, r, b, kind);
  else spmv_resid<T>(c.ex, M, nr, b, x, r, kind, layout);
}

// the finest level of Ã₃ in parity-split numbering (see SplitMap)
static SplitMap split_map(const stokes_ctx& c) {
  SplitMap sm;
  sm.m = 2 * c.lv[0].n - 1;
  sm.half = c.lv[0].n;
  return sm;
}
static double*& split_dinv_slot(Level& L, double*) { return L.A3_dinv_split64; }
static float*& split_dinv_slot(Level& L, float*) { return L.A3_dinv_split32; }
template <class T> static const T* split_dinv(stokes_ctx& c) {
  Level& L = c.lv[0];
  T*& slot = split_dinv_slot(L, (T*)nullptr);
  if (!slot) {
    slot = c.arena.alloc<T>(L.A3.rows);
    to_split<T>(c.ex, (size_t)L.A3.rows, 1, pick<T>(L.A3_dinv64, L.A3_dinv32), slot, false, split_map(c));
  }
  return slot;
}
// whether velocity V-cycles of A~_3 run their finest level split-numbered
// (option vcycle_split: 1 the interleaved lockstep cycles, 2 all)
template <class T> static bool use_split(const stokes_ctx& c, int which, bool il) {
  const bool wanted = c.opt.vcycle_split == 2 || (c.opt.vcycle_split == 1 && il);
  return wanted && which == 0 && c.lv.size() >= 2 && c.lv[0].A3.st != nullptr && stencil_in_use<T>(c.lv[0].A3, il);
}

// il: node-interleaved level vectors (K > 1); split: level 0 parity-split
// numbered (b, x and the temporaries of level 0)
template <class T>
static void vcycle(stokes_ctx& c, int which, int l, const T* b, T* x, bool xzero, int K, bool il, bool split) {
  SK_REQUIRE(which != 2 || K == 1, STOKES_ERR_ARG, "block V-cycle: one right-hand side per call");
  Level& L = c.lv[l];
  const int nr = (which == 1 ? 1 : 3) * K;
  const Csr& M = level_op(L, which);
  size_t len = (size_t)M.rows * nr;
  if (l + 1 == (int)c.lv.size()) {
    if (which == 2) {  // dense inverse over all 3 rows components
      dense_apply<T>(c.ex, pick<T>(L.AV_cinv64, L.AV_cinv32), 3 * M.rows, 1, b, x);
      return;
    }
    const T* Minv = which ? pick<T>(L.KQ_cinv64, L.KQ_cinv32) : pick<T>(L.A3_cinv64, L.A3_cinv32);
    dense_apply<T>(c.ex, Minv, M.rows, nr, b, x, il);
    return;
  }
  split = split && l == 0;
  const int layout = (il ? kLayoutIL : 0) | (split ? kLayoutSplit : 0);
  const SplitMap sm = split ? split_map(c) : SplitMap{};
  const T* dinv = which == 1 ? pick<T>(L.KQ_dinv64, L.KQ_dinv32)
                             : (which == 2 ? pick<T>(L.AV_dinv64, L.AV_dinv32)
                                           : (split ? split_dinv<T>(c) : pick<T>(L.A3_dinv64, L.A3_dinv32)));
  const double lhat = which == 1 ? L.KQ_lmax : (which == 2 ? L.AV_lmax : L.A3_lmax);
  double lmax = c.opt.cheb_high * lhat, lmin = c.opt.cheb_low * lhat;
  int deg = std::max(1, c.opt.cheb_degree);
  const int kind = which == 1 ? STOKES_KERNEL_SPMV_P1 : (l == 0 ? STOKES_KERNEL_SPMM_A3 : STOKES_KERNEL_SPMM_A3_COARSE);
  cheb_run<T>(c, M, nr, dinv, lmin, lmax, deg, b, x, xzero, kind, layout);
  Level& Lc = c.lv[l + 1];
  const Csr& Mc = level_op(Lc, which);
  size_t lenc = (size_t)Mc.rows * nr;
  // transfers from / to this level (the coarse level is always natural)
  auto restrict_to = [&](const T* r, T* bc) {
    if (split) restrict_split<T>(c.ex, L.R2, nr, r, bc, il, sm);
    else spmv_store<T>(c.ex, which == 1 ? L.R1 : L.R2, nr, r, bc, STOKES_KERNEL_TRANSFER, il);
  };
  auto prolong_into = [&](const T* xc, T* xf) {
    if (split) prolong_add_split<T>(c.ex, L.P2, nr, xc, xf, il, sm);
    else spmv_add<T>(c.ex, which == 1 ? L.P1 : L.P2, nr, xc, xf, STOKES_KERNEL_TRANSFER, il);
  };
  if (l == 0 && K == 1 && coarse_kernel_ok(c, which)) {
    MgProgram* P = mg_program<T>(c, which);
    {
      Tmp<T> r(c.pool, len);
      level_resid<T>(c, M, nr, b, x, r, kind, layout);
      restrict_to(r, (T*)P->b);
    }
    P->launch(c.ex);
    prolong_into((const T*)P->x, x);
  } else if (l == 0 && K == 1 && coarse_graph_ok(c, which)) {
    auto& G = c.cgraph[which][std::is_same<T, float>::value ? 1 : 0];
    if (!G.b) {
      G.b = c.arena.raw(lenc * sizeof(T));
      G.x = c.arena.raw(lenc * sizeof(T));
      G.pool.arena = &c.arena;
    }
    {
      Tmp<T> r(c.pool, len);
      level_resid<T>(c, M, nr, b, x, r, kind, layout);
      restrict_to(r, (T*)G.b);
    }
    coarse_run<T>(c, which, G);
    prolong_into((const T*)G.x, x);
  } else {
    Tmp<T> r(c.pool, len);
    level_resid<T>(c, M, nr, b, x, r, kind, layout);
    Tmp<T> bc(c.pool, lenc), xc(c.pool, lenc);
    restrict_to(r, bc);
    vcycle<T>(c, which, l + 1, bc, xc, true, K, il);
    prolong_into(xc, x);
  }
  cheb_run<T>(c, M, nr, dinv, lmin, lmax, deg, b, x, false, kind, layout);
}

// K > 1: the cycles run on node-interleaved copies (a row's 3K or K values
// contiguous, gathered as 16-byte vectors by the sparse kernels); b and x
// stay component-major K-blocks
// With a parity-split finest level (use_split) b is renumbered on the way in
// and x on the way out (one pass each, fused with the interleaving for K > 1).
template <class T> static void vcycles_plain(stokes_ctx& c, int which, const T* b, T* x, int cycles, int K = 1) {
  const bool il = K > 1;
  const bool split = use_split<T>(c, which, il);
  if (il || split) {
    const size_t rows = (size_t)level_op(c.lv[0], which).rows;
    const int nr = (which == 1 ? 1 : 3) * K;
    Tmp<T> bi(c.pool, rows * nr), xi(c.pool, rows * nr);
    if (split) to_split<T>(c.ex, rows, nr, b, bi, il, split_map(c));
    else to_interleaved<T>(c.ex, rows, nr, b, bi);
    vcycle<T>(c, which, 0, bi, xi, true, K, il, split);
    for (int k = 1; k < cycles; ++k) vcycle<T>(c, which, 0, bi, xi, false, K, il, split);
    if (split) from_split<T>(c.ex, rows, nr, xi, x, il, split_map(c));
    else to_component_major<T>(c.ex, rows, nr, xi, x);
    return;
  }
  vcycle<T>(c, which, 0, b, x, true, K);
  for (int k = 1; k < cycles; ++k) vcycle<T>(c, which, 0, b, x, false, K);
}

// A whole V-cycle in one graph needs every launch it makes to be untimed:
// allowed without profiling, or when the one timed class is not launched by
// a V-cycle of this kind.
constexpr size_t kMaxCycleGraphs = 128;
static bool cycle_graph_ok(const stokes_ctx& c, int which) {
  if (!c.opt.graphs || c.graphs_off || c.in_cycle_graph) return false;
  (void)which;
  return !c.prof.on || c.prof.only >= 0;
}

// Sync-free regions (a whole V-cycle; C with fixed inner iterations) from
// graphs keyed by their buffers: the first call with a key runs plainly
// (temporaries from the private pool), the second records the same sequence
// on the capture stream, later calls replay it on ex.s.
using GraphKey = std::tuple<int, int, const void*, void*, int>;
template <class Body> static void graph_region(stokes_ctx& c, const GraphKey& key, Body&& body) {
  auto it = c.vgraphs.find(key);
  if (it == c.vgraphs.end()) {
    if (c.vgraphs.size() >= kMaxCycleGraphs) {
      body();
      return;
    }
    it = c.vgraphs.emplace(key, stokes_ctx::CycleGraph{}).first;
  }
  auto& G = it->second;
  if (!c.vgraph_pool.arena) c.vgraph_pool.arena = &c.arena;
  if (!G.exec) {
    if (!c.cap_stream) SK_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    PoolSwap swap(c.pool, c.vgraph_pool);
    struct Flag {  // nested regions run plainly while this one is warmed or recorded
      bool& f;
      explicit Flag(bool& x) : f(x) { f = true; }
      ~Flag() { f = false; }
    } flag(c.in_cycle_graph);
    if (G.seen == 0) {
      body();
      G.seen = 1;
      return;
    }
    G.counts = Prof::Counts{};
    const cudaStream_t launch = c.ex.s;
    cudaGraph_t g = nullptr;
    SK_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    c.prof.capture = &G.counts;
    c.ex.s = c.cap_stream;
    try {
      body();
    } catch (const Error& err) {
      c.ex.s = launch;
      c.prof.capture = nullptr;
      cudaStreamEndCapture(c.cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      if (err.status != STOKES_ERR_CUDA) throw;
      // a step this runtime cannot record (the cooperative coarse-level
      // kernel): no more graphs for this context, run the region plainly
      (void)cudaGetLastError();
      c.graphs_off = true;
      c.vgraphs.erase(it);
      flag.f = false;
      body();
      return;
    } catch (...) {
      c.ex.s = launch;
      c.prof.capture = nullptr;
      cudaStreamEndCapture(c.cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    c.ex.s = launch;
    c.prof.capture = nullptr;
    SK_CUDA(cudaStreamEndCapture(c.cap_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    SK_CUDA(e);
  }
  SK_CUDA(cudaGraphLaunch(G.exec, c.ex.s));
  if (c.prof.on)
    for (int k = 0; k < STOKES_KERNEL_COUNT; ++k) {
      c.prof.rec[k].launches += G.counts.launches[k];
      c.prof.rec[k].bytes += G.counts.bytes[k];
    }
}

// K right-hand sides: b, x hold K blocks of the cycle's vector length
// (component-major, so the blocks are the 3K or K components of one sweep)
template <class T> static void vcycles(stokes_ctx& c, int which, const T* b, T* x, int cycles, int K = 1) {
  if (which == 2 && K > 1) {  // the 3x3-block operator takes one right-hand side per cycle
    const size_t len = 3 * (size_t)c.lv[0].nvi;
    for (int k = 0; k < K; ++k) vcycles<T>(c, which, b + k * len, x + k * len, cycles, 1);
    return;
  }
  if (!cycle_graph_ok(c, which)) {
    vcycles_plain<T>(c, which, b, x, cycles, K);
    return;
  }
  graph_region(c,
               GraphKey(which, (int)std::is_same<T, float>::value + 2 * (K - 1), (const void*)b, (void*)x, cycles),
               [&]() { vcycles_plain<T>(c, which, b, x, cycles, K); });
}

// ---------------------------------------------------------------------------
// preconditioned CG. The residual norm of step k is copied to the host while
// the preconditioner of step k+1 runs, so the GPU never idles on the check.
// ---------------------------------------------------------------------------
// fixed > 0: exactly `fixed` iterations and no host synchronisation at all.
// op(d, q, dq) computes q = M d and the device scalar *dq = d . q.
template <class T, class Op, class Pre>
static int pcg(stokes_ctx& c, size_t n, Op&& op, Pre&& pre, const T* b, T* x, double rtol, int maxit,
               bool* converged = nullptr, int fixed = 0) {
  Scalars& S = c.sc;
  const int s = S.take(5);
  double* D = S.d + s;  // 0,1: r.z (alternating), 2: d.q, 3: r.r, 4: b.b
  Tmp<T> r(c.pool, n), z(c.pool, n), d(c.pool, n), q(c.pool, n);
  zero<T>(c, x, n);
  copy<T>(c, r, b, n);
  double bn = 0.0;
  if (converged) *converged = true;
  if (fixed <= 0) {
    dot1<T>(c, (const T*)r, (const T*)r, n, D + 4, kDotFast);
    double bb = read_now(c, D + 4, s + 4);
    if (!std::isfinite(bb)) throw Error(STOKES_ERR_NAN, "non-finite right-hand side in an inner solve");
    if (bb == 0.0) {
      S.give(5);
      return 0;
    }
    bn = std::sqrt(bb);
  }
  pre((const T*)r, (T*)z);
  copy<T>(c, d, z, n);
  int irz = 0, irzn = 1;
  dot1<T>(c, (const T*)r, (const T*)z, n, D + irz, kDotFast);
  int it = 0;
  bool done = false;
  const int cap = fixed > 0 ? fixed : maxit;
  while (it < cap) {
    op((const T*)d, (T*)q, D + 2);
    ++it;
    if (fixed > 0) {
      cg_update<T>(c.ex, n, Coef::ratio(D + irz, D + 2), d, x, q, r);
      if (it == cap) {
        done = true;
        break;
      }
      pre((const T*)r, (T*)z);
    } else {
      cg_update_rr<T>(c.ex, c.ds, n, Coef::ratio(D + irz, D + 2), d, x, q, r, D + 3);  // and r . r
      read_issue(c, D + 3, s + 3);
      pre((const T*)r, (T*)z);
      double rr = read_wait(c, s + 3);
      if (!std::isfinite(rr)) throw Error(STOKES_ERR_NAN, "non-finite residual in an inner solve");
      if (std::sqrt(rr) <= rtol * bn) {
        done = true;
        break;
      }
    }
    dot1<T>(c, (const T*)r, (const T*)z, n, D + irzn, kDotFast);
    axpby<T>(c.ex, n, Coef::constant(1.0), z, Coef::cg_ratio(D + irzn, D + irz), d);
    std::swap(irz, irzn);
  }
  if (converged) *converged = done;
  S.give(5);
  return it;
}

// ---------------------------------------------------------------------------
// velocity operator and its inverse
// ---------------------------------------------------------------------------
// y = A x  (+ gamma mu B^T M_Q^{-1} B x for the augmented Lagrangian, Eq. def_of_Alambda)
template <class T> static void op_A(stokes_ctx& c, const T* x, T* y) {
  bsr3_apply<T>(c.ex, c.A, x, y, (const T*)nullptr);
  if (c.gamma > 0.0) {
    size_t np = npres(c);
    Tmp<T> bx(c.pool, np), mb(c.pool, np);
    b_apply<T>(c.ex, c.B, x, bx, (const T*)nullptr, 1.0);
    mass_inverse<T>(c, bx, mb, c.opt.mass_steps_al);
    bt_apply<T>(c.ex, c.Bt, mb, y, (const T*)nullptr, y, c.gamma * c.mu);
  }
}

// A^{-1} t by PCG preconditioned with `vcycles` V-cycles of A~_3 (Sec. 5.2:
// CG with (A~_{lambda,3})_2Vc)
template <class T> static int ainv(stokes_ctx& c, const T* t, T* w, double tol) {
  bool ok = true;
  int it = pcg<T>(
      c, nvel(c),
      [&](const T* x, T* y, double* dq) {
        if (c.gamma > 0.0) {
          op_A<T>(c, x, y);
          dot1<T>(c, x, (const T*)y, nvel(c), dq, kDotFast);
        } else {
          bsr3_apply_dot<T>(c.ex, c.A, x, y, c.ds, dq);  // d . A d fused into the product
        }
      },
      [&](const T* r, T* z) { vcycles<T>(c, velocity_cycle(c), r, z, std::max(1, c.opt.vcycles)); }, t, w, tol,
      c.opt.max_inner, &ok);
  c.inner_iters += it;
  if (!ok) c.inner_capped = true;
  return it;
}

// ---------------------------------------------------------------------------
// Cahouet-Chabard preconditioner (Eqs. Schur_complement_preconditioners):
//   C r = mu (1 + gamma) M_Q^{-1} r + dt^{-1} T^{-1} r,
//   T = B Lambda_V^{-1} B^T (C^Lambda) or L_Q (C^Delta), solved by PCG with one
//   V-cycle of eps M_Q + L_Q as preconditioner (Sec. 4.2), on the complement
//   of the constants.
// ---------------------------------------------------------------------------
template <class T> static int cprec_body(stokes_ctx& c, const T* r, T* z) {
  size_t np = npres(c), nv = nvel(c);
  Tmp<T> rp(c.pool, np), z1(c.pool, np), z2(c.pool, np);
  copy<T>(c, rp, r, np);
  project_mean<T>(c, rp, np, kDotFast);
  mass_inverse<T>(c, rp, z1, c.opt.mass_steps);
  const bool lumped = c.opt.schur_prec == STOKES_SCHUR_PREC_LUMPED;
  const bool vmass = c.opt.schur_prec == STOKES_SCHUR_PREC_MASS;
  const T* linv = pick<T>(c.lumped_inv64, c.lumped_inv32);
  int it = pcg<T>(
      c, np,
      [&](const T* p, T* y, double* dq) {
        if (lumped) {
          Tmp<T> t(c.pool, nv);
          bt_apply<T>(c.ex, c.Bt, p, t, linv, (const T*)nullptr, 1.0);
          b_apply<T>(c.ex, c.B, t, y, (const T*)nullptr, 1.0);
        } else if (vmass) {
          // B (M_V)_a^{-1} B^T p: a fixed Chebyshev polynomial in D^{-1} M_V
          // (symmetric positive definite, so PCG stays valid)
          Tmp<T> t(c.pool, nv), w(c.pool, nv);
          bt_apply<T>(c.ex, c.Bt, p, t, (const T*)nullptr, (const T*)nullptr, 1.0);
          cheb_run<T>(c, c.MV, 3, pick<T>(c.MV_dinv64, c.MV_dinv32), kMassVLow, kMassVHigh, c.opt.mass_steps_v, t,
                      w, true, STOKES_KERNEL_SPMM_A3);
          b_apply<T>(c.ex, c.B, w, y, (const T*)nullptr, 1.0);
        } else {
          spmv_store<T>(c.ex, c.LQ, 1, p, y, STOKES_KERNEL_SPMV_P1);
        }
        project_mean<T>(c, y, np, kDotFast);
        dot1<T>(c, p, (const T*)y, np, dq, kDotFast);
      },
      [&](const T* v, T* w) {
        Tmp<T> vp(c.pool, np);
        copy<T>(c, vp, v, np);
        project_mean<T>(c, vp, np, kDotFast);
        vcycles<T>(c, 1, vp, w, 1);
      },
      (const T*)rp, (T*)z2, c.opt.schur_inner_tol, c.opt.max_inner, nullptr, c.opt.schur_inner_iters);
  lincomb2<T>(c.ex, np, c.mu * (1.0 + c.gamma), z1, 1.0 / c.dt, z2, z);
  return it;
}

// With a fixed number of inner iterations C has no host synchronisation, so it
// is replayed from a graph (keyed by r, z and the device-scalar stack depth,
// whose slots it uses) when none of its launches is being timed per class.
static bool cprec_graph_ok(const stokes_ctx& c) {
  if (!c.opt.graphs || c.graphs_off || c.in_cycle_graph || c.opt.schur_inner_iters <= 0) return false;
  return !c.prof.on || c.prof.only >= 0;
}

template <class T> static void cprec(stokes_ctx& c, const T* r, T* z) {
  if (!cprec_graph_ok(c)) {
    c.schur_inner_iters += cprec_body<T>(c, r, z);
    return;
  }
  c.schur_inner_iters += c.opt.schur_inner_iters;  // fixed iterations: known without running
  graph_region(c, GraphKey(16 + (int)std::is_same<T, float>::value, 0, (const void*)r, (void*)z, c.sc.top),
               [&]() { (void)cprec_body<T>(c, r, z); });
}

// ---------------------------------------------------------------------------
// Method 1 on a residual system K [dU; dP] = [rF; rg]:
//   w = A_g^{-1} rF_g,  S dP = rg - B w  by flexible CG (Polak-Ribiere beta,
//   Notay 2000) preconditioned with C,  dU = w + sum_k alpha_k A_g^{-1} B^T d_k.
// With gamma > 0 the first block row is A_gamma dU - B^T dP = rF + gamma mu
// B^T M_Q^{-1} rg, which has the same solution (Eqs. LA_problem,
// Schur_LA_problem).
// ---------------------------------------------------------------------------
template <class T>
static void method1(stokes_ctx& c, const T* rF, const T* rg, T* dU, T* dP, double eta, double tol_in) {
  const size_t nv = nvel(c), np = npres(c);
  Tmp<T> Fg(c.pool, nv);
  const T* F = rF;
  if (c.gamma > 0.0) {
    Tmp<T> mg(c.pool, np);
    mass_inverse<T>(c, rg, mg, c.opt.mass_steps_al);
    bt_apply<T>(c.ex, c.Bt, mg, Fg, (const T*)nullptr, rF, c.gamma * c.mu);
    F = Fg;
  }
  ainv<T>(c, F, dU, tol_in);
  zero<T>(c, dP, np);
  Tmp<T> r(c.pool, np), z(c.pool, np), d(c.pool, np), q(c.pool, np), rold(c.pool, np);
  Tmp<T> t(c.pool, nv), wd(c.pool, nv);
  b_apply<T>(c.ex, c.B, dU, r, rg, -1.0);  // r = rg - B w
  project_mean<T>(c, r, np);
  Scalars& S = c.sc;
  const int s = S.take(6);
  double* D = S.d + s;  // 0,2: z.r (alternating) 1: d.q 3: z.r_old 4: r.r 5: beta numerator
  dot1<T>(c, (const T*)r, (const T*)r, np, D + 4, kDotExact);
  double rr0 = read_now(c, D + 4, s + 4);
  if (!std::isfinite(rr0)) throw Error(STOKES_ERR_NAN, "non-finite Schur right-hand side");
  if (rr0 == 0.0) {
    S.give(6);
    return;
  }
  cprec<T>(c, r, z);
  copy<T>(c, d, z, np);
  int irz = 0, irzn = 2;
  dot1<T>(c, (const T*)z, (const T*)r, np, D + irz, kDotExact);
  int k = 0;
  bool done = false;
  while (k < c.opt.max_outer) {
    bt_apply<T>(c.ex, c.Bt, d, t, (const T*)nullptr, (const T*)nullptr, 1.0);  // t = B^T d
    ainv<T>(c, t, wd, tol_in);                                                  // wd = A^{-1} t
    b_apply<T>(c.ex, c.B, wd, q, (const T*)nullptr, 1.0);                       // q = S d
    dot1<T>(c, (const T*)d, (const T*)q, np, D + 1, kDotExact);
    Coef alpha = Coef::ratio(D + irz, D + 1);
    cg_update<T>(c.ex, np, alpha, d, dP, (const T*)nullptr, (T*)nullptr);
    cg_update<T>(c.ex, nv, alpha, wd, dU, (const T*)nullptr, (T*)nullptr);
    copy<T>(c, rold, r, np);
    axpby<T>(c.ex, np, Coef::ratio(D + irz, D + 1, -1.0), q, Coef::constant(1.0), r);
    project_mean<T>(c, r, np);
    ++k;
    dot1<T>(c, (const T*)r, (const T*)r, np, D + 4, kDotExact);
    read_issue(c, D + 4, s + 4);
    cprec<T>(c, r, z);
    double rr = read_wait(c, s + 4);
    if (!std::isfinite(rr)) throw Error(STOKES_ERR_NAN, "non-finite Schur residual");
    if (std::sqrt(rr) <= eta * std::sqrt(rr0)) {
      done = true;
      break;
    }
    const T* xs[2] = {z, z};
    const T* ys[2] = {r, rold};
    double tmp2[1];
    (void)tmp2;
    dots<T>(c.ex, c.ds, 1, xs, ys, np, D + irzn, kDotExact);
    dots<T>(c.ex, c.ds, 1, xs + 1, ys + 1, np, D + 3, kDotExact);
    scalar_sub(c.ex, D + 5, D + irzn, D + 3);
    axpby<T>(c.ex, np, Coef::constant(1.0), z, Coef::cg_ratio(D + 5, D + irz), d);
    std::swap(irz, irzn);
  }
  c.outer_iters += k;
  if (!done) c.outer_capped = true;
  S.give(6);
}

// ---------------------------------------------------------------------------
// Method 2: right-preconditioned FGMRES(m) on the coupled system
//   [A_g  -B^T; B  0] (Sec. 2.4), preconditioner (Eq.
//   inexact_factorization_of_Alambda)
//   P^{-1} = [I  A~^{-1}B^T; 0 I] diag(A~^{-1}, C) [I 0; -B A~^{-1} I]
// or its block-triangular form without the left factor (Remark "Alternative
// preconditioner"). A~^{-1} = V-cycles of A~_3 or PCG on A_g to inner_tol.
// Arnoldi with classical Gram-Schmidt applied twice (CGS2), FP64 Hessenberg
// and Givens rotations on the host.
// ---------------------------------------------------------------------------
template <class T> static void atilde_inv(stokes_ctx& c, const T* r, T* z, double tol_in) {
  if (c.opt.m2_inner_cg)
    ainv<T>(c, r, z, tol_in);
  else
    vcycles<T>(c, velocity_cycle(c), r, z, std::max(1, c.opt.vcycles));
}

template <class T> static void block_prec(stokes_ctx& c, const T* ru, const T* rp, T* zu, T* zp, double tol_in) {
  const size_t nv = nvel(c), np = npres(c);
  Tmp<T> w(c.pool, nv), s(c.pool, np);
  atilde_inv<T>(c, ru, w, tol_in);                       // w = A~^{-1} ru
  b_apply<T>(c.ex, c.B, w, s, rp, -1.0);                 // s = rp - B w
  cprec<T>(c, s, zp);                                    // zp = C s
  if (c.opt.block_lu) {
    Tmp<T> t(c.pool, nv), v(c.pool, nv);
    bt_apply<T>(c.ex, c.Bt, zp, t, (const T*)nullptr, (const T*)nullptr, 1.0);
    atilde_inv<T>(c, t, v, tol_in);                      // v = A~^{-1} B^T zp
    lincomb2<T>(c.ex, nv, 1.0, w, 1.0, v, zu);           // zu = w + v
  } else {
    copy<T>(c, zu, (const T*)w, nv);
  }
}

template <class T>
static void method2(stokes_ctx& c, const T* rF, const T* rg, T* dU, T* dP, double eta, double tol_in) {
  const size_t nv = nvel(c), np = npres(c), N = nv + np;
  const int m = std::max(2, c.opt.restart);
  // Krylov basis V (m+1 vectors) and flexible basis Z (m vectors), each [u; p]
  std::vector<Tmp<T>*> V, Z;
  for (int j = 0; j <= m; ++j) V.push_back(new Tmp<T>(c.pool, N));
  for (int j = 0; j < m; ++j) Z.push_back(new Tmp<T>(c.pool, N));
  auto cleanup = [&]() {
    for (auto* p : V) delete p;
    for (auto* p : Z) delete p;
  };
  Scalars& S = c.sc;
  const int s = S.take(2 * (m + 1) + 2);
  double* D = S.d + s;
  try {
    Tmp<T> Fg(c.pool, nv);
    const T* F = rF;
    if (c.gamma > 0.0) {
      Tmp<T> mg(c.pool, np);
      mass_inverse<T>(c, rg, mg, c.opt.mass_steps_al);
      bt_apply<T>(c.ex, c.Bt, mg, Fg, (const T*)nullptr, rF, c.gamma * c.mu);
      F = Fg;
    }
    zero<T>(c, dU, nv);
    zero<T>(c, dP, np);
    // r0 = [F; rg]
    T* v0 = *V[0];
    copy<T>(c, v0, F, nv);
    copy<T>(c, v0 + nv, rg, np);
    project_mean<T>(c, v0 + nv, np);
    dot1<T>(c, (const T*)v0, (const T*)v0, N, D, kDotExact);
    double beta0 = std::sqrt(read_now(c, D, s));
    if (!std::isfinite(beta0)) throw Error(STOKES_ERR_NAN, "non-finite coupled right-hand side");
    double beta = beta0;
    int total = 0;
    bool done = beta0 == 0.0;
    std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1);
    while (!done && total < c.opt.max_outer) {
      scale_copy<T>(c.ex, N, Coef::constant(1.0 / beta), *V[0], *V[0]);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int j = 0;
      for (; j < m && total < c.opt.max_outer; ++j, ++total) {
        T* vj = *V[j];
        T* zj = *Z[j];
        T* w = *V[j + 1];
        block_prec<T>(c, vj, vj + nv, zj, zj + nv, tol_in);
        // w = K zj
        op_A<T>(c, zj, w);
        bt_apply<T>(c.ex, c.Bt, zj + nv, w, (const T*)nullptr, w, -1.0);
        b_apply<T>(c.ex, c.B, zj, w + nv, (const T*)nullptr, 1.0);
        // CGS2: two passes of h = V^T w (all basis vectors in one sweep that
        // reads w once), w -= V h (one sweep)
        for (int pass = 0; pass < 2; ++pass) {
          double* h = D + 2 + (pass ? m + 1 : 0);
          for (int i = 0; i <= j; i += kMaxBasis) {
            const int k = std::min(kMaxBasis, j + 1 - i);
            const T* vs[kMaxBasis];
            for (int t = 0; t < k; ++t) vs[t] = *V[i + t];
            mdot<T>(c.ex, c.ds, k, vs, w, N, h + i);
          }
          for (int i = 0; i <= j; i += kMaxBasis) {
            const int k = std::min(kMaxBasis, j + 1 - i);
            const T* vs[kMaxBasis];
            for (int t = 0; t < k; ++t) vs[t] = *V[i + t];
            maxpy<T>(c.ex, k, h + i, nullptr, -1.0, vs, w, N);
          }
        }
        dot1<T>(c, (const T*)w, (const T*)w, N, D + 1, kDotExact);
        SK_CUDA(cudaMemcpyAsync(S.h + s + 1, D + 1, sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost,
                                c.ex.s));
        host_sync(c);
        double hn = std::sqrt(S.h[s + 1]);
        for (int i = 0; i <= j; ++i) H[i * m + j] = S.h[s + 2 + i] + S.h[s + 2 + m + 1 + i];
        H[(j + 1) * m + j] = hn;
        if (!std::isfinite(hn)) throw Error(STOKES_ERR_NAN, "non-finite Arnoldi vector");
        if (hn > 0) scale_copy<T>(c.ex, N, Coef::constant(1.0 / hn), w, w);
        // Givens
        for (int i = 0; i < j; ++i) {
          double a = H[i * m + j], b = H[(i + 1) * m + j];
          H[i * m + j] = cs[i] * a + sn[i] * b;
          H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
        }
        double a = H[j * m + j], b = H[(j + 1) * m + j];
        double rden = std::hypot(a, b);
        cs[j] = rden > 0 ? a / rden : 1.0;
        sn[j] = rden > 0 ? b / rden : 0.0;
        H[j * m + j] = rden;
        H[(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        if (std::fabs(g[j + 1]) <= eta * beta0 || hn == 0.0) {
          ++j;
          ++total;
          done = true;
          break;
        }
      }
      // y = H^{-1} g (upper triangular j x j), x += Z y
      std::vector<double> y(j);
      for (int i = j - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < j; ++k) t -= H[i * m + k] * y[k];
        y[i] = t / H[i * m + i];
      }
      for (int i = 0; i < j; i += kMaxBasis) {  // [dU; dP] += Z y
        const int k = std::min(kMaxBasis, j - i);
        const T* zu[kMaxBasis];
        const T* zp[kMaxBasis];
        for (int t = 0; t < k; ++t) zu[t] = *Z[i + t], zp[t] = *Z[i + t] + nv;
        maxpy<T>(c.ex, k, nullptr, y.data() + i, 1.0, zu, dU, nv);
        maxpy<T>(c.ex, k, nullptr, y.data() + i, 1.0, zp, dP, np);
      }
      if (done || total >= c.opt.max_outer) break;
      // restart: r = [F; rg] - K x
      T* r0 = *V[0];
      op_A<T>(c, dU, r0);
      bt_apply<T>(c.ex, c.Bt, dP, r0, (const T*)nullptr, r0, -1.0);
      axpby<T>(c.ex, nv, Coef::constant(1.0), F, Coef::constant(-1.0), r0);
      b_apply<T>(c.ex, c.B, dU, r0 + nv, rg, -1.0);
      project_mean<T>(c, r0 + nv, np);
      dot1<T>(c, (const T*)r0, (const T*)r0, N, D, kDotExact);
      beta = std::sqrt(read_now(c, D, s));
      if (beta <= eta * beta0) done = true;
    }
    c.outer_iters += total;
    if (!done) c.outer_capped = true;
  } catch (...) {
    S.give(2 * (m + 1) + 2);
    cleanup();
    throw;
  }
  S.give(2 * (m + 1) + 2);
  cleanup();
}

// ---------------------------------------------------------------------------
// defect correction on the FP64 residual of the full system
// ---------------------------------------------------------------------------
template <class T>
static void correction(stokes_ctx& c, const double* rF, const double* rg, double* U, double* P, double eta,
                       double tol_in) {
  NvtxRange range(std::is_same<T, float>::value ? "correction pass (FP32)" : "correction pass (FP64)");
  const size_t nv = nvel(c), np = npres(c);
  Tmp<T> dU(c.pool, nv), dP(c.pool, np);
  const T* rFt;
  const T* rgt;
  Tmp<T> rF32(c.pool, std::is_same<T, double>::value ? 1 : nv), rg32(c.pool, std::is_same<T, double>::value ? 1 : np);
  if constexpr (std::is_same<T, double>::value) {
    rFt = rF;
    rgt = rg;
  } else {
    convert<double, float>(c.ex, nv, rF, rF32);
    convert<double, float>(c.ex, np, rg, rg32);
    rFt = rF32;
    rgt = rg32;
  }
  if (c.opt.method == STOKES_METHOD_COUPLED)
    method2<T>(c, rFt, rgt, dU, dP, eta, tol_in);
  else
    method1<T>(c, rFt, rgt, dU, dP, eta, tol_in);
  add_convert<T, double>(c.ex, nv, dU, U);
  add_convert<T, double>(c.ex, np, dP, P);
}

static int read_flag(stokes_ctx& c) {
  int flag = 0;
  SK_CUDA(cudaMemcpyAsync(&flag, c.d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.ex.s));
  host_sync(c);
  return flag;
}

// full residual rF = F - A U + B^T P, rg = g - B U and its relative norm
static double full_residual(stokes_ctx& c, const double* F, const double* g, const double* U, const double* P,
                            double* rF, double* rg, double normFg) {
  const size_t nv = nvel(c), np = npres(c);
  if (c.A.v32lo) {
    // mixed precision: the same FP64-accurate product on FP32 units
    Tmp<float> uh(c.pool, nv), ul(c.pool, nv);
    split_f64(c.ex, nv, U, uh, ul);
    bsr3_residual_df(c.ex, c.A, uh, ul, F, rF, STOKES_KERNEL_RESIDUAL);
  } else {
    bsr3_apply<double>(c.ex, c.A, U, rF, F, STOKES_KERNEL_RESIDUAL);
  }
  bt_apply<double>(c.ex, c.Bt, P, rF, (const double*)nullptr, rF, 1.0);
  b_apply<double>(c.ex, c.B, U, rg, g, -1.0);
  const int s = c.sc.take(2);
  const double* xs[2] = {rF, rg};
  dots<double>(c.ex, c.ds, 1, xs, xs, nv, c.sc.d + s);
  dots<double>(c.ex, c.ds, 1, xs + 1, xs + 1, np, c.sc.d + s + 1);
  SK_CUDA(cudaMemcpyAsync(c.sc.h + s, c.sc.d + s, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.ex.s));
  host_sync(c);
  double rr = c.sc.h[s] + c.sc.h[s + 1];
  c.sc.give(2);
  return std::sqrt(rr) / normFg;
}

// Solve K [U; P] = [F; g] in the reduced spaces (interior velocity, all P1
// nodes) to a true relative residual tol; P is normalised to int p_h = 0.
static int solve_reduced(stokes_ctx& c, const double* F, const double* g, double tol, double* U, double* P,
                         stokes_info* info, std::chrono::steady_clock::time_point t0) {
  const size_t nv = nvel(c), np = npres(c);
  c.outer_iters = c.inner_iters = c.schur_inner_iters = 0;
  c.outer_capped = c.inner_capped = false;
  SK_CUDA(cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.ex.s));
  Tmp<double> gz(c.pool, np), rF(c.pool, nv), rg(c.pool, np);
  const double* gp = g;
  if (!gp) {
    zero<double>(c, gz, np);
    gp = gz;
  }
  // compatibility of g: sum(g) = 0 (1^T B = 0)
  const int s = c.sc.take(3);
  {
    const double* xs[1] = {gp};
    dots<double>(c.ex, c.ds, 1, xs, (const double* const*)nullptr, np, c.sc.d + s);
    dots<double>(c.ex, c.ds, 1, xs, xs, np, c.sc.d + s + 1);
    const double* fs[1] = {F};
    dots<double>(c.ex, c.ds, 1, fs, fs, nv, c.sc.d + s + 2);
    SK_CUDA(cudaMemcpyAsync(c.sc.h + s, c.sc.d + s, 3 * sizeof(double), cudaMemcpyDeviceToHost, c.ex.s));
    host_sync(c);
  }
  double gsum = c.sc.h[s], gg = c.sc.h[s + 1], FF = c.sc.h[s + 2];
  c.sc.give(3);
  if (!std::isfinite(gsum) || !std::isfinite(gg) || !std::isfinite(FF))
    throw Error(STOKES_ERR_NAN, "non-finite right-hand side");
  if (std::fabs(gsum) > 1e-10 * std::sqrt((double)np * gg) + 1e-300)
    throw Error(STOKES_ERR_INCOMPATIBLE_RHS, "sum(g) must vanish for B u = g to be solvable");
  double normFg = std::sqrt(FF + gg);
  zero<double>(c, U, nv);
  zero<double>(c, P, np);
  int status = STOKES_OK;
  double rel = 0.0;
  int pass = 0;
  if (normFg > 0) {
   try {
    for (;; ++pass) {
      rel = full_residual(c, F, gp, U, P, rF, rg, normFg);
      if (!std::isfinite(rel)) {
        status = STOKES_ERR_NAN;
        break;
      }
      if (rel <= tol) break;
      if (pass >= c.opt.max_refine) {
        status = STOKES_ERR_NOT_CONVERGED;
        break;
      }
      // Pass schedule: each pass asks for a reduction of pass_tol and its inner
      // velocity solves for pass_tol / 30 (measured best on the 48^3 workload:
      // cheap passes, about three of them to reach 1e-8); the default for FP32
      // inner work. Otherwise one pass aims straight at tol with inner solves
      // at inner_tol (the paper's setting; the FP64 default).
      const bool passes = c.opt.pass_schedule == 1 || (c.opt.pass_schedule == 0 && c.mixed);
      double eta = passes ? std::max(c.opt.pass_tol, 0.5 * tol / rel) : std::max(0.5 * tol / rel, 1e-13);
      double tin = passes ? std::max(c.opt.inner_tol, c.opt.pass_tol / 30.0) : c.opt.inner_tol;
      if (c.mixed)
        correction<float>(c, rF, rg, U, P, eta, tin);
      else
        correction<double>(c, rF, rg, U, P, eta, tin);
    }
   } catch (const Error& e) {
    // a non-finite residual after a flagged breakdown is the breakdown
    if (e.status == STOKES_ERR_NAN && (read_flag(c) & 1))
      throw Error(STOKES_ERR_BREAKDOWN, std::string("Krylov breakdown (r^T z <= 0 or p^T A p <= 0), then ") + e.what());
    throw;
   }
  }
  // int p_h = 0: P -= (M_Q 1 . P) / (1^T M_Q 1)
  {
    const int s2 = c.sc.take(1);
    dot1<double>(c, (const double*)c.MQ1, (const double*)P, np, c.sc.d + s2);
    sub_mean<double>(c.ex, np, c.sc.d + s2, c.MQ1_sum, P);
    c.sc.give(1);
  }
  const int flag = read_flag(c);
  // a failed solve that met r^T z <= 0 or p^T A p <= 0 on the way broke down
  if ((status == STOKES_ERR_NOT_CONVERGED || status == STOKES_ERR_NAN) && (flag & 1)) status = STOKES_ERR_BREAKDOWN;
  if (flag & 4) status = STOKES_ERR_TIMEOUT;  // a bounded device wait expired
  if (info) {
    info->outer_iters = c.outer_iters;
    info->inner_iters = c.inner_iters;
    info->refinements = pass;
    info->status = status;
    info->rel_residual = rel;
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

int solve_context(stokes_ctx* cp, const double* f, const double* g, double tol, double* u, double* p,
                  stokes_info* info) {
  NvtxRange range("stokes_solve");
  stokes_ctx& c = *cp;
  auto t0 = std::chrono::steady_clock::now();
  c.sc.top = 0;
  const size_t nv = nvel(c), np = npres(c);
  Tmp<double> F(c.pool, nv);
  assemble_load(c.ex, c.n, c.lv[0].X, c.lv[0].A3, f, F, c.tet_vol);
  int status = solve_reduced(c, F, g, tol, c.U_last, c.P_last, info, t0);
  expand_velocity(c.ex, c.n, c.U_last, u);
  copy<double>(c, p, (const double*)c.P_last, np);
  host_sync(c);
  c.have_solution = true;
  if (info) info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

// ===========================================================================
// K right-hand sides in lockstep (stokes_solve_multi). The vectors below are
// K-vectors: the velocity blocks [K][nv] followed by the pressure blocks
// [K][np], or K plain blocks of one length. The V-cycles and Chebyshev mass
// inverses sweep each level matrix once for all K systems (3K or K
// component-major components), the K-RHS vector kernels serve all systems in
// one launch, and the A, B and B^T products run once per system. Every
// system keeps its own Krylov coefficients, Hessenberg matrix and
// convergence test; a converged system's vectors are zeroed and ride along.
// ===========================================================================
constexpr int kLockstep = 4;  // right-hand sides per lockstep group (3K and K components: 12 and 4)

static void read_k(stokes_ctx& c, const double* d, int slot, int count) {
  SK_CUDA(cudaMemcpyAsync(c.sc.h + slot, d, sizeof(double) * count, cudaMemcpyDeviceToHost, c.ex.s));
  host_sync(c);
}
static void read_k_issue(stokes_ctx& c, const double* d, int slot, int count) {
  SK_CUDA(cudaMemcpyAsync(c.sc.h + slot, d, sizeof(double) * count, cudaMemcpyDeviceToHost, c.ex.s));
  SK_CUDA(cudaEventRecord(c.ev_read, c.ex.s));
}
static unsigned all_bits(int K) { return K >= 32 ? ~0u : ((1u << K) - 1u); }
static bool has_bit(unsigned m, int k) { return (m >> k) & 1u; }

// r_k <- r_k - mean(r_k) for K plain blocks of length n
template <class T> static void project_mean_k(stokes_ctx& c, T* r, size_t n, int K) {
  const int s = c.sc.take(K);
  kdot<T>(c.ex, c.ds, n, 0, K, 1, r, (const T*)nullptr, c.sc.d + s);
  kaddconst<T>(c.ex, n, 0, K, 1, KCoefs::ratio(c.sc.d + s, nullptr, -1.0 / (double)n), r);
  c.sc.give(K);
}

// per-system B and B^T products: y_k = b_k + alpha B x_k; y_k = b_k + alpha s o (B^T x_k)
// (four systems: one product that reads the matrix once)
template <class T> static void b_apply_k(stokes_ctx& c, int K, const T* x, T* y, const T* b, double alpha) {
  const size_t nv = nvel(c), np = npres(c);
  if (K == 4) {
    b_apply<T>(c.ex, c.B, x, y, b, alpha, 4);
    return;
  }
  for (int k = 0; k < K; ++k) b_apply<T>(c.ex, c.B, x + k * nv, y + k * np, b ? b + k * np : nullptr, alpha);
}
template <class T>
static void bt_apply_k(stokes_ctx& c, int K, const T* x, T* y, const T* scale, const T* b, double alpha) {
  const size_t nv = nvel(c), np = npres(c);
  if (K == 4) {
    bt_apply<T>(c.ex, c.Bt, x, y, scale, b, alpha, 4);
    return;
  }
  for (int k = 0; k < K; ++k)
    bt_apply<T>(c.ex, c.Bt, x + k * np, y + k * nv, scale, b ? b + k * nv : nullptr, alpha);
}

// y_k = A_gamma x_k for K velocity blocks
template <class T> static void op_A_k(stokes_ctx& c, int K, const T* x, T* y) {
  const size_t nv = nvel(c), np = npres(c);
  bsr3_apply_k<T>(c.ex, c.A, K, x, y, (const T*)nullptr);
  if (c.gamma > 0.0) {
    Tmp<T> bx(c.pool, K * np), mb(c.pool, K * np);
    b_apply_k<T>(c, K, x, bx, (const T*)nullptr, 1.0);
    mass_inverse<T>(c, bx, mb, c.opt.mass_steps_al, K);
    bt_apply_k<T>(c, K, mb, y, (const T*)nullptr, y, c.gamma * c.mu);
  }
}

// Preconditioned CG on K systems of length n in lockstep (the same
// iteration as pcg() per system). fixed > 0: exactly `fixed` iterations, no
// host synchronisation. Otherwise a system stops updating (its coefficients
// masked to zero) once its residual meets rtol; the loop ends when all have.
// op(d, q, dq) computes q_k = M d_k and dq[k] = d_k . q_k.
template <class T, class Op, class Pre>
static int kpcg(stokes_ctx& c, size_t n, int K, Op&& op, Pre&& pre, const T* b, T* x, double rtol, int maxit,
                int fixed, unsigned* unconverged = nullptr) {
  Scalars& S = c.sc;
  const int s = S.take(5 * K);
  double* D = S.d + s;  // [0,K), [K,2K): r.z (alternating); [2K,3K): d.q; [3K,4K): r.r; [4K,5K): b.b
  const size_t len = (size_t)K * n;
  Tmp<T> r(c.pool, len), z(c.pool, len), d(c.pool, len), q(c.pool, len);
  zero<T>(c, x, len);
  copy<T>(c, r, b, len);
  unsigned act = all_bits(K);
  double bn[kMaxRhs] = {};
  if (fixed <= 0) {
    kdot<T>(c.ex, c.ds, n, 0, K, 1, r, r, D + 4 * K);
    read_k(c, D + 4 * K, s + 4 * K, K);
    for (int k = 0; k < K; ++k) {
      const double bb = S.h[s + 4 * K + k];
      if (!std::isfinite(bb)) {
        S.give(5 * K);
        throw Error(STOKES_ERR_NAN, "non-finite right-hand side in an inner solve");
      }
      if (bb == 0.0) act &= ~(1u << k);
      bn[k] = std::sqrt(bb);
    }
    if (!act) {
      S.give(5 * K);
      if (unconverged) *unconverged = 0;
      return 0;
    }
  }
  pre((const T*)r, (T*)z);
  copy<T>(c, d, z, len);
  int irz = 0, irzn = 1;
  kdot<T>(c.ex, c.ds, n, 0, K, 1, r, z, D + irz * K);
  int it = 0;
  const int cap = fixed > 0 ? fixed : maxit;
  try {
    while (it < cap) {
      op((const T*)d, (T*)q, D + 2 * K);
      ++it;
      KCoefs alpha = KCoefs::ratio(D + irz * K, D + 2 * K).mask(act);
      KCoefs malpha = KCoefs::ratio(D + irz * K, D + 2 * K, -1.0).mask(act);
      kaxpby<T>(c.ex, n, 0, K, 1, alpha, d, KCoefs::constant(1.0), x);
      kaxpby<T>(c.ex, n, 0, K, 1, malpha, q, KCoefs::constant(1.0), r);
      if (fixed > 0) {
        if (it == cap) break;
        pre((const T*)r, (T*)z);
      } else {
        kdot<T>(c.ex, c.ds, n, 0, K, 1, r, r, D + 3 * K);
        read_k_issue(c, D + 3 * K, s + 3 * K, K);
        pre((const T*)r, (T*)z);
        SK_CUDA(cudaEventSynchronize(c.ev_read));
        for (int k = 0; k < K; ++k) {
          if (!has_bit(act, k)) continue;
          const double rr = S.h[s + 3 * K + k];
          if (!std::isfinite(rr)) throw Error(STOKES_ERR_NAN, "non-finite residual in an inner solve");
          if (std::sqrt(rr) <= rtol * bn[k]) act &= ~(1u << k);
        }
        if (!act) break;
      }
      kdot<T>(c.ex, c.ds, n, 0, K, 1, r, z, D + irzn * K);
      kaxpby<T>(c.ex, n, 0, K, 1, KCoefs::constant(1.0), z, KCoefs::cg_ratio(D + irzn * K, D + irz * K).mask(act),
                d);
      std::swap(irz, irzn);
    }
  } catch (...) {
    S.give(5 * K);
    throw;
  }
  if (unconverged) *unconverged = fixed > 0 ? 0u : act;
  S.give(5 * K);
  return it;
}

// A^{-1} t for K velocity blocks by PCG with V-cycles (as ainv())
template <class T> static int ainv_k(stokes_ctx& c, int K, const T* t, T* w, double tol) {
  const size_t nv = nvel(c);
  unsigned left = 0;
  int it = kpcg<T>(
      c, nv, K,
      [&](const T* x, T* y, double* dq) {
        if (c.gamma > 0.0) {
          op_A_k<T>(c, K, x, y);
          kdot<T>(c.ex, c.ds, nv, 0, K, 1, x, (const T*)y, dq);
        } else {
          for (int k = 0; k < K; ++k) bsr3_apply_dot<T>(c.ex, c.A, x + k * nv, y + k * nv, c.ds, dq + k);
        }
      },
      [&](const T* r, T* z) { vcycles<T>(c, velocity_cycle(c), r, z, std::max(1, c.opt.vcycles), K); }, t, w, tol,
      c.opt.max_inner, 0, &left);
  c.inner_iters += it;
  if (left) c.inner_capped = true;
  return it;
}

// Cahouet-Chabard C for K pressure blocks (as cprec_body())
template <class T> static int cprec_body_k(stokes_ctx& c, int K, const T* r, T* z) {
  const size_t np = npres(c), nv = nvel(c), len = (size_t)K * np;
  Tmp<T> rp(c.pool, len), z1(c.pool, len), z2(c.pool, len);
  copy<T>(c, rp, r, len);
  project_mean_k<T>(c, rp, np, K);
  mass_inverse<T>(c, rp, z1, c.opt.mass_steps, K);
  const bool lumped = c.opt.schur_prec == STOKES_SCHUR_PREC_LUMPED;
  const bool vmass = c.opt.schur_prec == STOKES_SCHUR_PREC_MASS;
  const T* linv = pick<T>(c.lumped_inv64, c.lumped_inv32);
  int it = kpcg<T>(
      c, np, K,
      [&](const T* p, T* y, double* dq) {
        if (lumped) {
          Tmp<T> t(c.pool, (size_t)K * nv);
          bt_apply_k<T>(c, K, p, t, linv, (const T*)nullptr, 1.0);
          b_apply_k<T>(c, K, t, y, (const T*)nullptr, 1.0);
        } else if (vmass) {
          Tmp<T> t(c.pool, nv), w(c.pool, nv);
          for (int k = 0; k < K; ++k) {
            bt_apply<T>(c.ex, c.Bt, p + k * np, t, (const T*)nullptr, (const T*)nullptr, 1.0);
            cheb_run<T>(c, c.MV, 3, pick<T>(c.MV_dinv64, c.MV_dinv32), kMassVLow, kMassVHigh, c.opt.mass_steps_v, t,
                        w, true, STOKES_KERNEL_SPMM_A3);
            b_apply<T>(c.ex, c.B, w, y + k * np, (const T*)nullptr, 1.0);
          }
        } else {
          spmv_store<T>(c.ex, c.LQ, K, p, y, STOKES_KERNEL_SPMV_P1);
        }
        project_mean_k<T>(c, y, np, K);
        kdot<T>(c.ex, c.ds, np, 0, K, 1, p, (const T*)y, dq);
      },
      [&](const T* v, T* w) {
        Tmp<T> vp(c.pool, len);
        copy<T>(c, vp, v, len);
        project_mean_k<T>(c, vp, np, K);
        vcycles<T>(c, 1, vp, w, 1, K);
      },
      (const T*)rp, (T*)z2, c.opt.schur_inner_tol, c.opt.max_inner, c.opt.schur_inner_iters);
  lincomb2<T>(c.ex, len, c.mu * (1.0 + c.gamma), z1, 1.0 / c.dt, z2, z);
  return it;
}

template <class T> static void cprec_k(stokes_ctx& c, int K, const T* r, T* z) {
  if (!cprec_graph_ok(c)) {
    c.schur_inner_iters += cprec_body_k<T>(c, K, r, z);
    return;
  }
  c.schur_inner_iters += c.opt.schur_inner_iters;
  graph_region(c, GraphKey(16 + (int)std::is_same<T, float>::value, 100 + K, (const void*)r, (void*)z, c.sc.top),
               [&]() { (void)cprec_body_k<T>(c, K, r, z); });
}

template <class T> static void atilde_inv_k(stokes_ctx& c, int K, const T* r, T* z, double tol_in) {
  if (c.opt.m2_inner_cg)
    ainv_k<T>(c, K, r, z, tol_in);
  else
    vcycles<T>(c, velocity_cycle(c), r, z, std::max(1, c.opt.vcycles), K);
}

// the block preconditioner of method2 for K-vectors v -> z
template <class T> static void block_prec_k(stokes_ctx& c, int K, const T* v, T* z, double tol_in) {
  const size_t nv = nvel(c), np = npres(c), Kv = (size_t)K * nv;
  Tmp<T> w(c.pool, Kv), s(c.pool, (size_t)K * np);
  atilde_inv_k<T>(c, K, v, w, tol_in);            // w = A~^{-1} vu
  b_apply_k<T>(c, K, w, s, v + Kv, -1.0);         // s = vp - B w
  cprec_k<T>(c, K, s, z + Kv);                    // zp = C s
  if (c.opt.block_lu) {
    Tmp<T> t(c.pool, Kv), u(c.pool, Kv);
    bt_apply_k<T>(c, K, z + Kv, t, (const T*)nullptr, (const T*)nullptr, 1.0);
    atilde_inv_k<T>(c, K, t, u, tol_in);          // u = A~^{-1} B^T zp
    lincomb2<T>(c.ex, Kv, 1.0, w, 1.0, u, z);     // zu = w + u
  } else {
    copy<T>(c, z, (const T*)w, Kv);
  }
}

// Method 1 (flexible CG on the Schur complement, as method1()) for the K
// systems of the residual K-vector R into the K-vector X, in lockstep: each
// system keeps its own alpha, beta and stopping test; the inner A-solves run
// as one lockstep PCG whose systems stop on their own tolerances. A system
// that has converged gets a zero search direction, so its inner solves
// return at once. Arguments as method2_k().
template <class T>
static void method1_k(stokes_ctx& c, int K, const T* R, T* X, const double* eta, double tol_in, unsigned live,
                      int* its) {
  const size_t nv = nvel(c), np = npres(c), Kv = (size_t)K * nv, Kp = (size_t)K * np;
  T* dU = X;
  T* dP = X + Kv;
  const T* rg = R + Kv;
  Tmp<T> Fg(c.pool, c.gamma > 0.0 ? Kv : 1);
  const T* F = R;
  if (c.gamma > 0.0) {
    Tmp<T> mg(c.pool, Kp);
    mass_inverse<T>(c, rg, mg, c.opt.mass_steps_al, K);
    bt_apply_k<T>(c, K, mg, Fg, (const T*)nullptr, R, c.gamma * c.mu);
    F = Fg;
  }
  zero<T>(c, X, Kv + Kp);
  // systems left out get a zero right-hand side: their inner solves stop at once
  Tmp<T> Fl(c.pool, Kv);
  double keep[kMaxRhs] = {};
  for (int k = 0; k < K; ++k) keep[k] = has_bit(live, k) ? 1.0 : 0.0;
  kaxpby<T>(c.ex, nv, 0, K, 1, KCoefs::host(keep, K), F, KCoefs::constant(0.0), Fl);
  ainv_k<T>(c, K, Fl, dU, tol_in);
  Tmp<T> r(c.pool, Kp), z(c.pool, Kp), d(c.pool, Kp), q(c.pool, Kp), rold(c.pool, Kp);
  Tmp<T> t(c.pool, Kv), wd(c.pool, Kv);
  b_apply_k<T>(c, K, dU, r, rg, -1.0);  // r = rg - B w
  project_mean_k<T>(c, r, np, K);
  Scalars& S = c.sc;
  const int s = S.take(6 * K);
  struct Give {
    Scalars& S;
    int n;
    ~Give() { S.give(n); }
  } give{S, 6 * K};
  double* D = S.d + s;  // [0,K), [2K,3K): z.r (alternating); [K,2K): d.q; [3K,4K): z.r_old; [4K,5K): r.r;
                        // [5K,6K): beta numerators
  kdot<T>(c.ex, c.ds, np, 0, K, 1, r, r, D + 4 * K);
  read_k(c, D + 4 * K, s + 4 * K, K);
  double rr0[kMaxRhs] = {};
  unsigned act = live;
  for (int k = 0; k < K; ++k) {
    rr0[k] = S.h[s + 4 * K + k];
    if (!std::isfinite(rr0[k])) throw Error(STOKES_ERR_NAN, "non-finite Schur right-hand side");
    if (rr0[k] == 0.0) act &= ~(1u << k);
  }
  if (!act) return;
  cprec_k<T>(c, K, r, z);
  kaxpby<T>(c.ex, np, 0, K, 1, KCoefs::constant(1.0).mask(act), z, KCoefs::constant(0.0), d);
  int irz = 0, irzn = 2;
  kdot<T>(c.ex, c.ds, np, 0, K, 1, z, r, D + irz * K);
  int it = 0;
  while (it < c.opt.max_outer) {
    bt_apply_k<T>(c, K, d, t, (const T*)nullptr, (const T*)nullptr, 1.0);  // t = B^T d
    ainv_k<T>(c, K, t, wd, tol_in);                                         // wd = A^{-1} t
    b_apply_k<T>(c, K, wd, q, (const T*)nullptr, 1.0);                      // q = S d
    kdot<T>(c.ex, c.ds, np, 0, K, 1, d, q, D + K);
    KCoefs alpha = KCoefs::ratio(D + irz * K, D + K).mask(act);
    kaxpby<T>(c.ex, np, 0, K, 1, alpha, d, KCoefs::constant(1.0), dP);
    kaxpby<T>(c.ex, nv, 0, K, 1, alpha, wd, KCoefs::constant(1.0), dU);
    copy<T>(c, rold, r, Kp);
    kaxpby<T>(c.ex, np, 0, K, 1, KCoefs::ratio(D + irz * K, D + K, -1.0).mask(act), q, KCoefs::constant(1.0), r);
    project_mean_k<T>(c, r, np, K);
    ++it;
    for (int k = 0; k < K; ++k)
      if (has_bit(act, k)) ++its[k];
    kdot<T>(c.ex, c.ds, np, 0, K, 1, r, r, D + 4 * K);
    read_k_issue(c, D + 4 * K, s + 4 * K, K);
    cprec_k<T>(c, K, r, z);
    SK_CUDA(cudaEventSynchronize(c.ev_read));
    for (int k = 0; k < K; ++k) {
      if (!has_bit(act, k)) continue;
      const double rr = S.h[s + 4 * K + k];
      if (!std::isfinite(rr)) throw Error(STOKES_ERR_NAN, "non-finite Schur residual");
      if (std::sqrt(rr) <= eta[k] * std::sqrt(rr0[k])) act &= ~(1u << k);
    }
    if (!act) break;
    kdot<T>(c.ex, c.ds, np, 0, K, 1, z, r, D + irzn * K);
    kdot<T>(c.ex, c.ds, np, 0, K, 1, z, rold, D + 3 * K);
    ksub(c.ex, K, D + 5 * K, D + irzn * K, D + 3 * K);  // Polak-Ribiere numerator
    // d = z + beta d for the systems still iterating, 0 for the others
    kaxpby<T>(c.ex, np, 0, K, 1, KCoefs::constant(1.0).mask(act), z, KCoefs::cg_ratio(D + 5 * K, D + irz * K).mask(act),
              d);
    std::swap(irz, irzn);
  }
  c.outer_iters += it;
  if (act) c.outer_capped = true;
}

// Method 2 (right-preconditioned FGMRES(m), CGS2) for the K systems of the
// residual K-vector R (rF blocks, then rg blocks) into the K-vector X, in
// lockstep: one Arnoldi step of every live system per iteration, one host
// read per iteration for all of them. eta[k]: relative reduction wanted of
// system k; `live`: the systems to solve (others get X_k = 0); its[k] counts
// the iterations system k took part in.
template <class T>
static void method2_k(stokes_ctx& c, int K, const T* R, T* X, const double* eta, double tol_in, unsigned live,
                      int* its) {
  const size_t nv = nvel(c), np = npres(c), Kv = (size_t)K * nv, KN = (size_t)K * (nv + np);
  const int m = std::max(2, c.opt.restart);
  const int ld = m + 1;
  std::vector<std::unique_ptr<Tmp<T>>> V, Z;
  for (int j = 0; j <= m; ++j) V.emplace_back(new Tmp<T>(c.pool, KN));
  for (int j = 0; j < m; ++j) Z.emplace_back(new Tmp<T>(c.pool, KN));
  Scalars& S = c.sc;
  const int nsl = K * (2 * ld + 2);
  const int s = S.take(nsl);
  struct Give {
    Scalars& S;
    int n;
    ~Give() { S.give(n); }
  } give{S, nsl};
  double* D = S.d + s;                 // [0,K): norms
  double* h0 = D + K;                  // [K][ld]: first Gram-Schmidt pass
  double* h1 = D + K + K * ld;         // [K][ld]: second pass
  double* ww = D + K + 2 * K * ld;     // [K]: w . w
  const double* H0 = S.h + s + K;
  const double* H1 = S.h + s + K + K * ld;
  const double* WW = S.h + s + K + 2 * K * ld;
  Tmp<T> Fg(c.pool, c.gamma > 0.0 ? Kv : 1);
  const T* F = R;
  const T* rg = R + Kv;
  if (c.gamma > 0.0) {
    Tmp<T> mg(c.pool, (size_t)K * np);
    mass_inverse<T>(c, rg, mg, c.opt.mass_steps_al, K);
    bt_apply_k<T>(c, K, mg, Fg, (const T*)nullptr, R, c.gamma * c.mu);
    F = Fg;
  }
  zero<T>(c, X, KN);
  T* v0 = *V[0];
  copy<T>(c, v0, F, Kv);
  copy<T>(c, v0 + Kv, rg, (size_t)K * np);
  project_mean_k<T>(c, v0 + Kv, np, K);
  kdot<T>(c.ex, c.ds, nv, np, K, 3, v0, v0, D);
  read_k(c, D, s, K);
  double beta0[kMaxRhs] = {}, beta[kMaxRhs] = {};
  for (int k = 0; k < K; ++k) {
    beta0[k] = beta[k] = std::sqrt(S.h[s + k]);
    if (!std::isfinite(beta0[k])) throw Error(STOKES_ERR_NAN, "non-finite coupled right-hand side");
    if (beta0[k] == 0.0) live &= ~(1u << k);
  }
  int total = 0;
  std::vector<double> H((size_t)K * ld * m), cs((size_t)K * m), sn((size_t)K * m), g((size_t)K * ld), y(m);
  std::vector<double> coef((size_t)K * kMaxBasisK);
  int jk[kMaxRhs] = {};
  while (live && total < c.opt.max_outer) {
    double scl[kMaxRhs] = {};
    for (int k = 0; k < K; ++k) scl[k] = has_bit(live, k) ? 1.0 / beta[k] : 0.0;
    kaxpby<T>(c.ex, nv, np, K, 3, KCoefs::host(scl, K), *V[0], KCoefs::constant(0.0), *V[0]);
    std::fill(g.begin(), g.end(), 0.0);
    for (int k = 0; k < K; ++k) g[(size_t)k * ld] = beta[k], jk[k] = 0;
    unsigned act = live, conv = 0;
    int j = 0;
    for (; j < m && total < c.opt.max_outer; ++j, ++total) {
      T* vj = *V[j];
      T* zj = *Z[j];
      T* w = *V[j + 1];
      block_prec_k<T>(c, K, vj, zj, tol_in);
      op_A_k<T>(c, K, zj, w);                                           // w = K zj
      bt_apply_k<T>(c, K, zj + Kv, w, (const T*)nullptr, w, -1.0);
      b_apply_k<T>(c, K, zj, w + Kv, (const T*)nullptr, 1.0);
      for (int pass = 0; pass < 2; ++pass) {                           // CGS2
        double* h = pass ? h1 : h0;
        const T* vs[kMaxBasisK];
        for (int i = 0; i <= j; i += kMaxBasisK) {
          const int kk = std::min(kMaxBasisK, j + 1 - i);
          for (int t = 0; t < kk; ++t) vs[t] = *V[i + t];
          kmdot<T>(c.ex, c.ds, nv, np, K, kk, vs, w, h + i, ld);
        }
        for (int i = 0; i <= j; i += kMaxBasisK) {
          const int kk = std::min(kMaxBasisK, j + 1 - i);
          for (int t = 0; t < kk; ++t) vs[t] = *V[i + t];
          kmaxpy<T>(c.ex, nv, np, K, kk, vs, h + i, nullptr, ld, -1.0, w);
        }
      }
      kdot<T>(c.ex, c.ds, nv, np, K, 3, w, w, ww);
      read_k(c, D, s, nsl);
      double wscale[kMaxRhs] = {};
      for (int k = 0; k < K; ++k) {
        if (!has_bit(act, k)) continue;
        ++its[k];
        double* Hk = H.data() + (size_t)k * ld * m;
        double* ck = cs.data() + (size_t)k * m;
        double* sk_ = sn.data() + (size_t)k * m;
        double* gk = g.data() + (size_t)k * ld;
        const double hn = std::sqrt(WW[k]);
        if (!std::isfinite(hn)) throw Error(STOKES_ERR_NAN, "non-finite Arnoldi vector");
        for (int i = 0; i <= j; ++i) Hk[i * m + j] = H0[k * ld + i] + H1[k * ld + i];
        Hk[(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {  // Givens
          const double a = Hk[i * m + j], b = Hk[(i + 1) * m + j];
          Hk[i * m + j] = ck[i] * a + sk_[i] * b;
          Hk[(i + 1) * m + j] = -sk_[i] * a + ck[i] * b;
        }
        const double a = Hk[j * m + j], b = Hk[(j + 1) * m + j];
        const double rden = std::hypot(a, b);
        ck[j] = rden > 0 ? a / rden : 1.0;
        sk_[j] = rden > 0 ? b / rden : 0.0;
        Hk[j * m + j] = rden;
        Hk[(j + 1) * m + j] = 0.0;
        gk[j + 1] = -sk_[j] * gk[j];
        gk[j] = ck[j] * gk[j];
        jk[k] = j + 1;
        if (std::fabs(gk[j + 1]) <= eta[k] * beta0[k] || hn == 0.0) {
          act &= ~(1u << k);
          conv |= 1u << k;
        } else {
          wscale[k] = 1.0 / hn;
        }
      }
      // next basis vector: w_k / |w_k| for systems still iterating, 0 for the rest
      kaxpby<T>(c.ex, nv, np, K, 3, KCoefs::host(wscale, K), w, KCoefs::constant(0.0), w);
      if (!act) {
        ++j;
        ++total;
        break;
      }
    }
    // X_k += Z y_k, y_k = H_k^{-1} g_k over the jk[k] columns system k built
    int jmax = 0;
    for (int k = 0; k < K; ++k)
      if (has_bit(live, k)) jmax = std::max(jmax, jk[k]);
    std::vector<double> Y((size_t)K * m, 0.0);
    for (int k = 0; k < K; ++k) {
      if (!has_bit(live, k)) continue;
      const double* Hk = H.data() + (size_t)k * ld * m;
      const double* gk = g.data() + (size_t)k * ld;
      double* yk = Y.data() + (size_t)k * m;
      for (int i = jk[k] - 1; i >= 0; --i) {
        double t = gk[i];
        for (int q = i + 1; q < jk[k]; ++q) t -= Hk[i * m + q] * yk[q];
        yk[i] = t / Hk[i * m + i];
      }
    }
    for (int i = 0; i < jmax; i += kMaxBasisK) {
      const int kk = std::min(kMaxBasisK, jmax - i);
      const T* zs[kMaxBasisK];
      for (int t = 0; t < kk; ++t) zs[t] = *Z[i + t];
      for (int k = 0; k < K; ++k)
        for (int t = 0; t < kk; ++t) coef[(size_t)k * kk + t] = Y[(size_t)k * m + i + t];
      kmaxpy<T>(c.ex, nv, np, K, kk, zs, nullptr, coef.data(), kk, 1.0, X);
    }
    live &= ~conv;
    if (!live || total >= c.opt.max_outer) break;
    // restart: r = [F; rg] - K X
    T* r0 = *V[0];
    op_A_k<T>(c, K, X, r0);
    bt_apply_k<T>(c, K, X + Kv, r0, (const T*)nullptr, r0, -1.0);
    axpby<T>(c.ex, Kv, Coef::constant(1.0), F, Coef::constant(-1.0), r0);
    b_apply_k<T>(c, K, X, r0 + Kv, rg, -1.0);
    project_mean_k<T>(c, r0 + Kv, np, K);
    kdot<T>(c.ex, c.ds, nv, np, K, 3, r0, r0, D);
    read_k(c, D, s, K);
    for (int k = 0; k < K; ++k) {
      if (!has_bit(live, k)) continue;
      beta[k] = std::sqrt(S.h[s + k]);
      if (!std::isfinite(beta[k])) throw Error(STOKES_ERR_NAN, "non-finite coupled residual");
      if (beta[k] <= eta[k] * beta0[k]) live &= ~(1u << k);
    }
  }
  c.outer_iters += total;
  if (live) c.outer_capped = true;
}

// full FP64 residuals of K systems: R = [F - A U + B^T P; g - B U] (K-vectors
// of the solutions X), rel[k] = |R_k| / normFg[k]
static void full_residual_k(stokes_ctx& c, int K, const double* F, const double* g, const double* X, double* R,
                            const double* normFg, double* rel) {
  const size_t nv = nvel(c), np = npres(c), Kv = (size_t)K * nv;
  if (K == 4 && c.A.v32lo && c.A.sym && c.A.sym->v32lo) {  // one sweep of each matrix for the four
    Tmp<float> uh(c.pool, Kv), ul(c.pool, Kv);
    split_f64(c.ex, Kv, X, uh, ul);
    {
      // values hi + lo once; per right-hand side x hi + lo, b and y (FP64)
      ProfScope ps(c.ex, STOKES_KERNEL_RESIDUAL, 8.0 * (double)c.A.sym->total + 4.0 * 3.0 * nvi_of(c) * 24.0);
      sym3_residual_df4(c.ex, c.A, uh, ul, F, R);
    }
    bt_apply<double>(c.ex, c.Bt, X + Kv, R, (const double*)nullptr, R, 1.0, 4);
    b_apply<double>(c.ex, c.B, X, R + Kv, g, -1.0, 4);
  } else {
   for (int k = 0; k < K; ++k) {
    const double* Uk = X + k * nv;
    double* rFk = R + k * nv;
    if (c.A.v32lo) {
      Tmp<float> uh(c.pool, nv), ul(c.pool, nv);
      split_f64(c.ex, nv, Uk, uh, ul);
      bsr3_residual_df(c.ex, c.A, uh, ul, F + k * nv, rFk, STOKES_KERNEL_RESIDUAL);
    } else {
      bsr3_apply<double>(c.ex, c.A, Uk, rFk, F + k * nv, STOKES_KERNEL_RESIDUAL);
    }
    bt_apply<double>(c.ex, c.Bt, X + Kv + k * np, rFk, (const double*)nullptr, rFk, 1.0);
    b_apply<double>(c.ex, c.B, Uk, R + Kv + k * np, g + k * np, -1.0);
   }
  }
  const int s = c.sc.take(K);
  kdot<double>(c.ex, c.ds, nv, np, K, 3, R, R, c.sc.d + s);
  read_k(c, c.sc.d + s, s, K);
  for (int k = 0; k < K; ++k) rel[k] = normFg[k] > 0 ? std::sqrt(c.sc.h[s + k]) / normFg[k] : 0.0;
  c.sc.give(K);
}

template <class T>
static void correction_k(stokes_ctx& c, int K, const double* R, double* X, const double* eta, double tol_in,
                         unsigned live, int* its) {
  NvtxRange range(std::is_same<T, float>::value ? "lockstep correction pass (FP32)" : "lockstep correction pass (FP64)");
  const size_t KN = (size_t)K * (nvel(c) + npres(c));
  Tmp<T> dX(c.pool, KN);
  Tmp<T> R32(c.pool, std::is_same<T, double>::value ? 1 : KN);
  const T* Rt;
  if constexpr (std::is_same<T, double>::value) {
    Rt = R;
  } else {
    convert<double, float>(c.ex, KN, R, R32);
    Rt = R32;
  }
  if (c.opt.method == STOKES_METHOD_COUPLED)
    method2_k<T>(c, K, Rt, dX, eta, tol_in, live, its);
  else
    method1_k<T>(c, K, Rt, dX, eta, tol_in, live, its);
  add_convert<T, double>(c.ex, KN, dX, X);
}

// K systems K [U_k; P_k] = [F_k; g_k] in the reduced spaces (as
// solve_reduced()): F [K][nv], g [K][np] or null, solutions into the
// K-vector X; info[k] and the returned status per system in status[k].
static void solve_reduced_k(stokes_ctx& c, int K, const double* F, const double* g, double tol, double* X,
                            stokes_info* info, int* status, std::chrono::steady_clock::time_point t0) {
  const size_t nv = nvel(c), np = npres(c), Kv = (size_t)K * nv, KN = (size_t)K * (nv + np);
  c.outer_iters = c.inner_iters = c.schur_inner_iters = 0;
  c.outer_capped = c.inner_capped = false;
  SK_CUDA(cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.ex.s));
  Tmp<double> gz(c.pool, (size_t)K * np), R(c.pool, KN);
  const double* gp = g;
  if (!gp) {
    zero<double>(c, gz, (size_t)K * np);
    gp = gz;
  }
  double normFg[kMaxRhs] = {}, rel[kMaxRhs] = {};
  {
    const int s = c.sc.take(3 * K);
    kdot<double>(c.ex, c.ds, np, 0, K, 1, gp, (const double*)nullptr, c.sc.d + s);
    kdot<double>(c.ex, c.ds, np, 0, K, 1, gp, gp, c.sc.d + s + K);
    kdot<double>(c.ex, c.ds, nv, 0, K, 1, F, F, c.sc.d + s + 2 * K);
    read_k(c, c.sc.d + s, s, 3 * K);
    for (int k = 0; k < K; ++k) {
      const double gsum = c.sc.h[s + k], gg = c.sc.h[s + K + k], FF = c.sc.h[s + 2 * K + k];
      if (!std::isfinite(gsum) || !std::isfinite(gg) || !std::isfinite(FF)) {
        c.sc.give(3 * K);
        throw Error(STOKES_ERR_NAN, "non-finite right-hand side");
      }
      if (std::fabs(gsum) > 1e-10 * std::sqrt((double)np * gg) + 1e-300) {
        c.sc.give(3 * K);
        throw Error(STOKES_ERR_INCOMPATIBLE_RHS, "sum(g) must vanish for B u = g to be solvable");
      }
      normFg[k] = std::sqrt(FF + gg);
    }
    c.sc.give(3 * K);
  }
  zero<double>(c, X, KN);
  unsigned pending = 0;
  int refinements[kMaxRhs] = {}, its[kMaxRhs] = {};
  for (int k = 0; k < K; ++k) {
    status[k] = STOKES_OK;
    if (normFg[k] > 0) pending |= 1u << k;
  }
  try {
    for (int pass = 0; pending; ++pass) {
      full_residual_k(c, K, F, gp, X, R, normFg, rel);
      double eta[kMaxRhs] = {};
      const bool passes = c.opt.pass_schedule == 1 || (c.opt.pass_schedule == 0 && c.mixed);
      for (int k = 0; k < K; ++k) {
        if (!has_bit(pending, k)) continue;
        refinements[k] = pass;
        if (!std::isfinite(rel[k])) {
          status[k] = STOKES_ERR_NAN;
          pending &= ~(1u << k);
        } else if (rel[k] <= tol) {
          pending &= ~(1u << k);
        } else if (pass >= c.opt.max_refine) {
          status[k] = STOKES_ERR_NOT_CONVERGED;
          pending &= ~(1u << k);
        }
        eta[k] = passes ? std::max(c.opt.pass_tol, 0.5 * tol / rel[k]) : std::max(0.5 * tol / rel[k], 1e-13);
      }
      if (!pending) break;
      const double tin = passes ? std::max(c.opt.inner_tol, c.opt.pass_tol / 30.0) : c.opt.inner_tol;
      if (c.mixed)
        correction_k<float>(c, K, R, X, eta, tin, pending, its);
      else
        correction_k<double>(c, K, R, X, eta, tin, pending, its);
    }
  } catch (const Error& e) {
    if (e.status == STOKES_ERR_NAN && (read_flag(c) & 1))
      throw Error(STOKES_ERR_BREAKDOWN, std::string("Krylov breakdown (r^T z <= 0 or p^T A p <= 0), then ") + e.what());
    throw;
  }
  // int p_h = 0 per system
  {
    const int s2 = c.sc.take(1);
    for (int k = 0; k < K; ++k) {
      double* Pk = X + Kv + k * np;
      dot1<double>(c, (const double*)c.MQ1, (const double*)Pk, np, c.sc.d + s2);
      sub_mean<double>(c.ex, np, c.sc.d + s2, c.MQ1_sum, Pk);
    }
    c.sc.give(1);
  }
  const int flag = read_flag(c);
  for (int k = 0; k < K; ++k) {
    if ((status[k] == STOKES_ERR_NOT_CONVERGED || status[k] == STOKES_ERR_NAN) && (flag & 1))
      status[k] = STOKES_ERR_BREAKDOWN;
    if (flag & 4) status[k] = STOKES_ERR_TIMEOUT;
    if (info) {
      info[k].outer_iters = its[k];
      info[k].inner_iters = c.inner_iters;
      info[k].refinements = refinements[k];
      info[k].status = status[k];
      info[k].rel_residual = rel[k];
      info[k].solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
  }
}

// K forces f [K][(2n+1)^3][3] -> u [K][(2n+1)^3][3], p [K][(n+1)^3]: groups
// of kLockstep systems in lockstep (a short last group is padded with zero
// systems; a single one takes the one-system path).
int solve_multi_context(stokes_ctx* cp, int K, const double* f, const double* g, double tol, double* u, double* p,
                        stokes_info* info) {
  NvtxRange range("stokes_solve_multi");
  stokes_ctx& c = *cp;
  auto t0 = std::chrono::steady_clock::now();
  c.sc.top = 0;
  const size_t nv = nvel(c), np = npres(c);
  const size_t Nall = 3 * (size_t)(2 * c.n + 1) * (2 * c.n + 1) * (2 * c.n + 1);
  int worst = STOKES_OK;
  auto note = [&](int st) {
    if (worst == STOKES_OK && st != STOKES_OK) worst = st;
  };
  for (int k0 = 0; k0 < K;) {
    const int left = K - k0;
    if (left == 1) {
      note(solve_context(cp, f + k0 * Nall, g ? g + k0 * np : nullptr, tol, u + k0 * Nall, p + k0 * np,
                         info ? info + k0 : nullptr));
      ++k0;
      continue;
    }
    const int kb = std::min(kLockstep, left), W = kLockstep;
    Tmp<double> F(c.pool, (size_t)W * nv), X(c.pool, (size_t)W * (nv + np));
    Tmp<double> G(c.pool, g ? (size_t)W * np : 1);
    for (int k = 0; k < kb; ++k) assemble_load(c.ex, c.n, c.lv[0].X, c.lv[0].A3, f + (k0 + k) * Nall, F + k * nv, c.tet_vol);
    if (kb < W) zero<double>(c, F + kb * nv, (size_t)(W - kb) * nv);
    if (g) {
      copy<double>(c, G, g + k0 * np, (size_t)kb * np);
      if (kb < W) zero<double>(c, G + kb * np, (size_t)(W - kb) * np);
    }
    stokes_info inf[kLockstep] = {};
    int st[kLockstep] = {};
    solve_reduced_k(c, W, F, g ? (const double*)G : nullptr, tol, X, inf, st, t0);
    for (int k = 0; k < kb; ++k) {
      expand_velocity(c.ex, c.n, X + k * nv, u + (k0 + k) * Nall);
      copy<double>(c, p + (k0 + k) * np, (const double*)(X + (size_t)W * nv + k * np), np);
      if (info) info[k0 + k] = inf[k];
      note(st[k]);
    }
    // the last system's solution serves a following stokes_adjoint
    copy<double>(c, c.U_last, (const double*)(X + (kb - 1) * nv), nv);
    copy<double>(c, c.P_last, (const double*)(X + (size_t)W * nv + (kb - 1) * np), np);
    c.have_solution = true;
    k0 += kb;
  }
  host_sync(c);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info)
    for (int k = 0; k < K; ++k) info[k].solve_ms = ms;
  return worst;
}

// Adjoint. K = [A -B^T; B 0] has K^T = [A B^T; -B 0]; with lp = -P' the
// transposed system K^T [lu; lp] = [jU; jP] is the forward system
// K [lu; P'] = [jU; -jP]. J depends on the normalised pressure, so jP is first
// projected with (I - m 1^T / 1^T m)^T, m = M_Q 1, which makes sum(jP) = 0.
// Then dJ/dF = lu, dJ/dg = lp, dJ/df = M_V^T lu (all nodes), and
// dJ/dmu = -lu^T (dA/dmu) U = -lu^T E_V U, with E_V U = (A U - M_V U / dt) / mu
// (the augmented-Lagrangian form has the same solution for every gamma).
int adjoint_context(stokes_ctx* cp, const double* dJdu, const double* dJdp, double tol, double* dJdf,
                    double* dJdg, double* dJdmu, stokes_info* info) {
  NvtxRange range("stokes_adjoint");
  stokes_ctx& c = *cp;
  auto t0 = std::chrono::steady_clock::now();
  const size_t nv = nvel(c), np = npres(c);
  Tmp<double> jU(c.pool, nv), jP(c.pool, np), lu(c.pool, nv), lp(c.pool, np);
  restrict_velocity(c.ex, c.n, dJdu, jU);
  if (dJdp) {
    // jP <- -(jP - m (1.jP) / (1.m))  (projected and negated)
    const int s = c.sc.take(1);
    copy<double>(c, jP, dJdp, np);
    dot1<double>(c, (const double*)jP, (const double*)nullptr, np, c.sc.d + s);
    Tmp<double> t(c.pool, np);
    scale_copy<double>(c.ex, np, Coef::ratio(c.sc.d + s, nullptr, 1.0 / c.MQ1_sum), c.MQ1, t);
    lincomb2<double>(c.ex, np, -1.0, jP, 1.0, t, jP);
    c.sc.give(1);
  } else {
    zero<double>(c, jP, np);
  }
  int status = solve_reduced(c, jU, jP, tol, lu, lp, info, t0);
  // dJ/df = M_V^T lu on all nodes
  assemble_load_transpose(c.ex, c.n, c.lv[0].X, lu, dJdf);
  if (dJdg) scale_copy<double>(c.ex, np, Coef::constant(-1.0), lp, dJdg);
  if (dJdmu) {
    Tmp<double> AU(c.pool, nv), MU(c.pool, nv);
    size_t N = (size_t)(2 * c.n + 1) * (2 * c.n + 1) * (2 * c.n + 1);
    Tmp<double> Uall(c.pool, 3 * N);
    bsr3_apply<double>(c.ex, c.A, c.U_last, AU, (const double*)nullptr);
    expand_velocity(c.ex, c.n, c.U_last, Uall);
    assemble_load(c.ex, c.n, c.lv[0].X, c.lv[0].A3, Uall, MU, c.tet_vol);
    lincomb2<double>(c.ex, nv, 1.0 / c.mu, AU, -1.0 / (c.mu * c.dt), MU, AU);  // E_V U
    const int s = c.sc.take(1);
    dot1<double>(c, (const double*)lu, (const double*)AU, nv, c.sc.d + s);
    *dJdmu = -read_now(c, c.sc.d + s, s);
    c.sc.give(1);
  }
  host_sync(c);
  if (info) info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

// ---------------------------------------------------------------------------
// operator access for tests (FP64)
// ---------------------------------------------------------------------------
void apply_operator(stokes_ctx* cp, int op, int level, const double* x, double* y) {
  stokes_ctx& c = *cp;
  SK_REQUIRE(level >= 0 && level < (int)c.lv.size(), STOKES_ERR_ARG, "level out of range");
  const Level& L = c.lv[level];
  if (op != STOKES_OP_A3 && op != STOKES_OP_KQ && op != STOKES_OP_VCYCLE_A3 && op != STOKES_OP_PROLONG_P2 &&
      op != STOKES_OP_RESTRICT_P2 && op != STOKES_OP_PROLONG_P1)
    SK_REQUIRE(level == 0, STOKES_ERR_ARG, "operator defined on level 0 only");
  const size_t np = npres(c), nv = nvel(c);
  switch (op) {
    case STOKES_OP_A: bsr3_apply<double>(c.ex, c.A, x, y, nullptr); break;
    case STOKES_OP_A3: spmv_store<double>(c.ex, L.A3, 3, x, y, STOKES_KERNEL_SPMM_A3); break;
    case STOKES_OP_B: b_apply<double>(c.ex, c.B, x, y, nullptr, 1.0); break;
    case STOKES_OP_BT: bt_apply<double>(c.ex, c.Bt, x, y, nullptr, nullptr, 1.0); break;
    case STOKES_OP_MQ: spmv_store<double>(c.ex, c.MQ, 1, x, y, STOKES_KERNEL_SPMV_P1); break;
    case STOKES_OP_LQ: spmv_store<double>(c.ex, c.LQ, 1, x, y, STOKES_KERNEL_SPMV_P1); break;
    case STOKES_OP_KQ: spmv_store<double>(c.ex, L.KQ, 1, x, y, STOKES_KERNEL_SPMV_P1); break;
    case STOKES_OP_LUMPED_INV: {
      // y = Lambda^{-1} x per node and component
      Tmp<double> ones(c.pool, 1);
      (void)ones;
      SK_CUDA(cudaMemcpyAsync(y, x, nv * sizeof(double), cudaMemcpyDeviceToDevice, c.ex.s));
      cheb_first<double>(c.ex, nv, 3, c.lumped_inv64, x, 1.0, y, y);
      break;
    }
    case STOKES_OP_VCYCLE_A3: {
      SK_REQUIRE(level == 0, STOKES_ERR_ARG, "V-cycle from level 0 only");
      vcycles<double>(c, 0, x, y, std::max(1, c.opt.vcycles));
      break;
    }
    case STOKES_OP_VCYCLE_KQ: vcycles<double>(c, 1, x, y, 1); break;
    case STOKES_OP_VCYCLE_VEL:
      SK_REQUIRE(level == 0, STOKES_ERR_ARG, "V-cycle from level 0 only");
      vcycles<double>(c, velocity_cycle(c), x, y, std::max(1, c.opt.vcycles));
      break;
    case STOKES_OP_SCHUR_PREC: cprec<double>(c, x, y); break;
    case STOKES_OP_SCHUR: {
      Tmp<double> t(c.pool, nv), w(c.pool, nv);
      bt_apply<double>(c.ex, c.Bt, x, t, nullptr, nullptr, 1.0);
      ainv<double>(c, t, w, c.opt.inner_tol);
      b_apply<double>(c.ex, c.B, w, y, nullptr, 1.0);
      break;
    }
    case STOKES_OP_AGAMMA: op_A<double>(c, x, y); break;
    case STOKES_OP_PROLONG_P2:
      SK_REQUIRE(level + 1 < (int)c.lv.size(), STOKES_ERR_ARG, "no coarser level");
      spmv_store<double>(c.ex, L.P2, 3, x, y, STOKES_KERNEL_TRANSFER);
      break;
    case STOKES_OP_RESTRICT_P2:
      SK_REQUIRE(level + 1 < (int)c.lv.size(), STOKES_ERR_ARG, "no coarser level");
      spmv_store<double>(c.ex, L.R2, 3, x, y, STOKES_KERNEL_TRANSFER);
      break;
    case STOKES_OP_PROLONG_P1:
      SK_REQUIRE(level + 1 < (int)c.lv.size(), STOKES_ERR_ARG, "no coarser level");
      spmv_store<double>(c.ex, L.P1, 1, x, y, STOKES_KERNEL_TRANSFER);
      break;
    case STOKES_OP_LOAD: assemble_load(c.ex, c.n, c.lv[0].X, c.lv[0].A3, x, y, c.tet_vol); break;
    case STOKES_OP_A_DF: {
      SK_REQUIRE(c.A.v32lo, STOKES_ERR_ARG, "double-float A needs a mixed-precision context");
      Tmp<float> xh(c.pool, nv), xl(c.pool, nv);
      Tmp<double> zero_b(c.pool, nv);
      zero<double>(c, zero_b, nv);
      split_f64(c.ex, nv, x, xh, xl);
      Tmp<double> t(c.pool, nv);
      bsr3_residual_df(c.ex, c.A, xh, xl, zero_b, t, STOKES_KERNEL_RESIDUAL);  // t = -A x
      scale_copy<double>(c.ex, nv, Coef::constant(-1.0), t, y);
      break;
    }
    default: throw Error(STOKES_ERR_ARG, "unknown operator");
  }
  (void)np;
  host_sync(c);
}

// ---------------------------------------------------------------------------
// setup helpers that need the solver kernels
// ---------------------------------------------------------------------------
// lambda_max(D^{-1} M) from the Lanczos tridiagonal of `steps` Jacobi-PCG
// steps (the CG coefficients give the Lanczos matrix; Golub & Van Loan 10.2).
double estimate_lmax(stokes_ctx& c, const Csr& M, const double* dinv, int steps, uint64_t seed) {
  const size_t n = (size_t)M.rows * M.br;  // 3x3 blocks: all components, component-major
  if (n == 0) return 1.0;
  std::vector<double> hb(n);
  uint64_t st = seed * 0x9E3779B97F4A7C15ULL + 1;
  for (size_t i = 0; i < n; ++i) {
    st += 0x9E3779B97F4A7C15ULL;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    hb[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
  Tmp<double> r(c.pool, n), z(c.pool, n), d(c.pool, n), q(c.pool, n), tmp(c.pool, n);
  SK_CUDA(cudaMemcpyAsync(r, hb.data(), n * sizeof(double), cudaMemcpyHostToDevice, c.ex.s));
  const int s = c.sc.take(3);
  double* D = c.sc.d + s;
  cheb_first<double>(c.ex, n, 1, dinv, r, 1.0, z, tmp);
  copy<double>(c, d, z, n);
  dot1<double>(c, (const double*)r, (const double*)z, n, D);
  double rz = read_now(c, D, s);
  std::vector<double> al, be;
  for (int j = 0; j < steps; ++j) {
    if (M.br == 3) bsr3_apply<double>(c.ex, M, d, q, nullptr, -1);
    else spmv_store<double>(c.ex, M, 1, d, q, -1);
    dot1<double>(c, (const double*)d, (const double*)q, n, D + 1);
    double dq = read_now(c, D + 1, s + 1);
    if (!(dq > 0) || !(rz > 0)) break;
    double a = rz / dq;
    cg_update<double>(c.ex, n, Coef::constant(a), d, tmp, q, r);
    cheb_first<double>(c.ex, n, 1, dinv, r, 1.0, z, tmp);
    dot1<double>(c, (const double*)r, (const double*)z, n, D + 2);
    double rzn = read_now(c, D + 2, s + 2);
    double b = rzn / rz;
    al.push_back(a);
    be.push_back(b);
    axpby<double>(c.ex, n, Coef::constant(1.0), z, Coef::constant(b), d);
    rz = rzn;
    if (!(rz > 0)) break;
  }
  c.sc.give(3);
  int k = (int)al.size();
  SK_REQUIRE(k > 0, STOKES_ERR_ARG, "spectrum estimate failed (matrix not positive definite?)");
  std::vector<double> dg(k), off(k > 1 ? k - 1 : 1);
  for (int j = 0; j < k; ++j) {
    dg[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < k) off[j] = std::sqrt(be[j]) / al[j];
  }
  // largest eigenvalue of the symmetric tridiagonal by Sturm bisection
  double hi = 0;
  for (int j = 0; j < k; ++j)
    hi = std::max(hi, dg[j] + (j > 0 ? std::fabs(off[j - 1]) : 0) + (j + 1 < k ? std::fabs(off[j]) : 0));
  double lo = 0;
  auto count_below = [&](double x) {
    int cnt = 0;
    double q = 1.0;
    for (int j = 0; j < k; ++j) {
      q = dg[j] - x - (j > 0 ? off[j - 1] * off[j - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 100; ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= k) hi = mid; else lo = mid;
  }
  return hi;
}

}  // namespace sk
