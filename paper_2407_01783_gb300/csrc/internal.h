// Internal declarations of the GB300 generalized-Stokes library.
// Host orchestration (solver.cu, capi.cu) talks to the kernels (assembly.cu,
// sparse.cu, blas1.cu) only through the launch wrappers declared here.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <map>
#include <memory>
#include <tuple>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/stokes.h"

namespace sk {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define SK_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      throw ::sk::Error(e_ == cudaErrorMemoryAllocation ? STOKES_ERR_OOM           \
                                                        : STOKES_ERR_CUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)
#define SK_CHECK_LAUNCH() SK_CUDA(cudaGetLastError())
#define SK_REQUIRE(cond, st, msg) \
  do {                            \
    if (!(cond)) throw ::sk::Error((st), (msg)); \
  } while (0)

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// An NVTX range for the lifetime of the object (solver phases show up as
// named ranges under a profiler; without one attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// profiling: CUDA events around launches of one kernel class
// ---------------------------------------------------------------------------
struct Prof {
  bool on = false;
  int only = -1;  // >= 0: CUDA events only around launches of this class (all are counted)
  // launches recorded into a CUDA graph are counted here instead (no events)
  struct Counts {
    double bytes[STOKES_KERNEL_COUNT] = {};
    int64_t launches[STOKES_KERNEL_COUNT] = {};
  };
  Counts* capture = nullptr;
  struct Rec {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    double bytes = 0;        // all launches (graph replays included)
    int64_t launches = 0;
    double ev_bytes = 0;     // the launches bracketed by events
    int64_t ev_launches = 0;
  } rec[STOKES_KERNEL_COUNT];
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void reset();
  ~Prof();
};

struct Exec {
  cudaStream_t s = nullptr;
  Prof* prof = nullptr;
  int* flag = nullptr;  // per-context status bits set by kernels (1: Krylov breakdown,
                        // 4: a bounded device wait expired)
};

// Brackets one launch with events when profiling is on.
struct ProfScope {
  Exec ex;
  int kind;
  cudaEvent_t e1 = nullptr;
  ProfScope(const Exec& e, int k, double bytes);
  ~ProfScope();
};

// ---------------------------------------------------------------------------
// Stencil-structured storage of a matrix on a Kuhn level. Every row node's
// neighbours follow one of 8 fixed stencils (by the parity class of its
// half-grid coordinates; P1 nodes have a single class), so a row needs no
// column indices: column = row + lin[e] for stencil entry e when the neighbour
// lies inside the index space, else the entry is absent (stored as 0). Each
// class's entry list is padded with zero entries (offset 0) to a multiple of
// kStencilVec, and the values of class c are stored
// [e / kStencilVec][row-in-class][e % kStencilVec]: one vector load gives a
// thread the weights of kStencilVec entries, and a warp of consecutive
// same-class rows reads one contiguous segment per load.
// ---------------------------------------------------------------------------
constexpr int kMaxStencil = 256;
constexpr int kStencilVec = 4;
// Rows of one class along x are grouped by kStencilRows per thread; the value
// layout pads each class's x-extent to a multiple of kStencilRows so that the
// values of a thread's rows are one aligned vector.
constexpr int kStencilRows = 1;
struct StencilOp {
  int p2 = 1;                // 1: interior P2 index space, 0: P1 index space
  int n = 0;
  int ncls = 0;
  int rows[8] = {}, ext[8][3] = {}, q0[8][3] = {}, S[8] = {}, dbeg[8] = {};
  int Sreal[8] = {};                // entries before padding to a multiple of kStencilVec
  int pext[8] = {}, prows[8] = {};  // padded x-extent and padded row count per class
  long long voff[8] = {};
  long long total = 0;       // stored entries (all classes, padding included)
  long long total_real = 0;  // stored entries without the padding entries
  signed char d[kMaxStencil][3] = {};  // half-grid offsets of entry e
  int lin[kMaxStencil] = {};           // linear index offsets of entry e
  int lin_split[kMaxStencil] = {};     // the same in parity-split numbering (P2 only, see SplitMap)
  int nd = 0;
  double* v64 = nullptr;
  float* v32 = nullptr;
  template <class T> T* v() const;
};
template <> inline double* StencilOp::v<double>() const { return v64; }
template <> inline float* StencilOp::v<float>() const { return v32; }

// Kernel-side view of a StencilOp (passed by value; blocks of one class are
// contiguous: class c owns blocks [bbeg[c], bbeg[c+1])).
struct StArgs {
  int p2, n, ncls, lo, hi, m, R;  // R: rows per thread of the launch using these args
  int split;                      // rows and columns in parity-split numbering (P2 only)
  int rows[8], ext[8][3], q0[8][3], S[8], Sreal[8], dbeg[8], pext[8], prows[8];
  long long voff[8];
  int bbeg[9];
  signed char d[kMaxStencil][3];
  int lin[kMaxStencil];
};
StArgs stencil_args(const StencilOp& s, int block, int rows_per_thread, bool split = false);

// Parity-split numbering of the interior P2 nodes of a level (m = 2n - 1
// points per axis): within every x-line the nodes of even x-index t come
// first (t / 2), then those of odd t (n + t / 2); y and z strides unchanged.
// The rows of one stencil class share the parity of t, so the neighbours a
// warp of consecutive class rows gathers are consecutive words instead of
// every second one. The map of a natural index i:
struct SplitMap {
  int m = 0, half = 0;  // points per axis; nodes of even t per line (n)
#ifdef __CUDACC__
  __host__ __device__ __forceinline__ int operator()(int i) const {
    const int t = i % m;
    return i - t + ((t & 1) ? half + (t >> 1) : (t >> 1));
  }
#endif
};

#ifdef __CUDACC__
// class and row-in-class of this thread; false if past the class end
// class c and thread-in-class t; each thread owns a.R consecutive padded
// rows of one x-line: padded row index pr = t * a.R
__device__ __forceinline__ bool st_locate(const StArgs& a, int& c, int& t) {
  c = 0;
#pragma unroll 1
  while (c + 1 < a.ncls && (int)blockIdx.x >= a.bbeg[c + 1]) ++c;
  t = ((int)blockIdx.x - a.bbeg[c]) * (int)blockDim.x + (int)threadIdx.x;
  return t * a.R < a.prows[c];
}
// padded row pr -> x index i (may be >= ext: padding) and coordinates
__device__ __forceinline__ void st_coords(const StArgs& a, int c, int pr, int& i, int& qx, int& qy, int& qz) {
  const int px = a.pext[c], ey = a.ext[c][1];
  i = pr % px;
  qx = a.q0[c][0] + 2 * i;
  qy = a.q0[c][1] + 2 * ((pr / px) % ey);
  qz = a.q0[c][2] + 2 * (pr / (px * ey));
}
// index of half-grid node q in the matrix's index space
__device__ __forceinline__ int st_index(const StArgs& a, int qx, int qy, int qz) {
  if (a.p2) {
    const int t = qx - 1;
    const int xs = a.split ? ((t & 1) ? a.n + (t >> 1) : (t >> 1)) : t;
    return xs + a.m * ((qy - 1) + a.m * (qz - 1));
  }
  return (qx >> 1) + a.m * ((qy >> 1) + a.m * (qz >> 1));
}
__device__ __forceinline__ bool st_inside(const StArgs& a, int qx, int qy, int qz) {
  return qx >= a.lo && qx <= a.hi && qy >= a.lo && qy <= a.hi && qz >= a.lo && qz <= a.hi;
}
#endif

// ---------------------------------------------------------------------------
// double-float BSR3 residual. Error-free transformations (published methods):
// TwoProduct with an FMA, p + e = a * b exactly (Ogita, Rump & Oishi 2005);
// TwoSum, s + e = a + b exactly (Knuth, TAOCP vol. 2, 4.2.2). The _rn
// intrinsics keep the compiler from contracting these steps into FMAs.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
struct DF {
  float h, l;
};
// s += (ah + al) * (xh + xl), dropping al * xl (2^-48 relative)
__device__ __forceinline__ void df_madd(DF& s, float ah, float al, float xh, float xl) {
  const float ph = __fmul_rn(ah, xh);
  const float pe = __fmaf_rn(ah, xh, -ph);
  const float pc = __fmaf_rn(ah, xl, __fmul_rn(al, xh));
  const float t = __fadd_rn(s.h, ph);
  const float z = __fsub_rn(t, s.h);
  const float e = __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, z)), __fsub_rn(ph, z));
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(e, __fadd_rn(pe, pc)));
}
// s += a * b with both rounding errors kept (the Dot2 step of Ogita, Rump &
// Oishi 2005: TwoProduct by FMA, then TwoSum): a dot product of FP32 vectors
// as accurate as if accumulated in twice the working precision, on FP32 units
__device__ __forceinline__ void df_dot(DF& s, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s.h, p);
  const float z = __fsub_rn(t, s.h);
  const float e = __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, z)), __fsub_rn(p, z));
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(e, pe));
}
__device__ __forceinline__ void df_add(DF& s, float oh, float ol) {
  const float t = __fadd_rn(s.h, oh);
  const float z = __fsub_rn(t, s.h);
  const float e = __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, z)), __fsub_rn(oh, z));
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(ol, e));
}
#endif

// ---------------------------------------------------------------------------
// Symmetric stencil storage of a 3x3-block operator on the interior P2 nodes
// (the strain-form A). Rows are grouped by the 8 parity classes of the P2
// stencil storage; a row stores only its diagonal block and the blocks of its
// "upper" neighbours (offset lexicographically positive in (z, y, x)). The
// block of a "lower" neighbour j = i + o is A(j, i)^T, read from row j's
// storage (class cs = class(i) XOR parity(o), entry -o), so every stored value
// is read twice per product and the matrix bytes are halved. Values of class c
// are stored [entry][9][row-in-class] (row-major 3x3 blocks), so a warp of
// consecutive same-class rows reads 128 contiguous bytes per block entry.
// ---------------------------------------------------------------------------
constexpr int kMaxSym = 160;
struct Sym3Op {
  int n = 0;
  int rows[8] = {}, ext[8][3] = {}, q0[8][3] = {}, pext[8] = {}, prows[8] = {};
  int ubeg[9] = {};                   // class c: upper entries (diagonal first) [ubeg[c], ubeg[c+1])
  signed char ud[kMaxSym][3] = {};    // half-grid offset of upper entry
  int ulin[kMaxSym] = {};             // linear index offset of upper entry
  long long voff[8] = {};             // class c: block e, entry k at voff[c] + (9 e + k) prows[c] + row
  int lbeg[9] = {};                   // class c: lower entries [lbeg[c], lbeg[c+1])
  signed char ld[kMaxSym][3] = {};    // half-grid offset o of lower entry (neighbour j = i + o)
  int llin[kMaxSym] = {};
  int lcls[kMaxSym] = {};             // class of j
  long long lbase[kMaxSym] = {};      // voff[class j] + 9 * (entry -o of class j) * prows[class j]
  signed char ldel[kMaxSym][3] = {};  // position of j in its class minus position of i in its class
  long long total = 0;                // stored values (9 per stored block)
  int group = 1;                      // threads per row of the products (1, 2, 4 or 8)
  int batch = 8;                      // entries whose loads a lane issues together (2, 4 or 8)
  double* v64 = nullptr;
  float* v32 = nullptr;
  float* v32lo = nullptr;             // FP32(v64 - v32): double-float residual
  template <class T> T* v() const;
};
template <> inline double* Sym3Op::v<double>() const { return v64; }
template <> inline float* Sym3Op::v<float>() const { return v32; }

// ---------------------------------------------------------------------------
// sparse matrices: CSR over (possibly) small dense blocks, values stored as
// br*bc planes of nnz entries each (plane j at v + j*nnz) so that consecutive
// lanes read consecutive addresses.
// ---------------------------------------------------------------------------
struct Csr {
  int rows = 0, cols = 0;
  long long nnz = 0;
  int br = 1, bc = 1;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  float* v32lo = nullptr;  // v64 - v32 rounded to FP32 (double-float residual), or null
  int group = 8;  // threads per row
  int group4 = 0; // threads per row of four-right-hand-side products (B, B^T; 0: group)
  const StencilOp* st = nullptr;  // same matrix in stencil storage (used when set, see st_min_single)
  int st_min_single = 0;          // component-major products (one right-hand side) use the stencil
                                  // storage only on matrices with at least this many rows
  const Sym3Op* sym = nullptr;    // 3x3-block matrix in symmetric stencil storage: used for the
                                  // double-float residual, and for all products if sym_products
  bool sym_products = false;
  template <class T> T* v() const;
  double bytes(int elem) const {  // algorithmic bytes of one product (matrix only)
    return (double)nnz * (4.0 + elem * br * bc) + 4.0 * (rows + 1);
  }
};
template <> inline double* Csr::v<double>() const { return v64; }
template <> inline float* Csr::v<float>() const { return v32; }

// Device allocations owned by a context.
struct Arena {
  std::vector<void*> ptrs;
  void* raw(size_t bytes);
  template <class T> T* alloc(size_t n) { return (T*)raw(sizeof(T) * (n ? n : 1)); }
  void free_all();
};

// Reusable device vectors keyed by (element size, length): after the first
// solve no further allocation happens.
struct VecPool {
  Arena* arena = nullptr;
  std::unordered_map<uint64_t, std::vector<void*>> free_;
  void* get(size_t elems, int esz);
  void put(void* p, size_t elems, int esz);
};

template <class T> struct Tmp {
  VecPool* pool;
  size_t n;
  T* p;
  Tmp(VecPool& vp, size_t n_) : pool(&vp), n(n_), p((T*)vp.get(n_, sizeof(T))) {}
  ~Tmp() { pool->put(p, n, sizeof(T)); }
  Tmp(const Tmp&) = delete;
  Tmp& operator=(const Tmp&) = delete;
  operator T*() const { return p; }
};

// Device-resident FP64 scalars used by Krylov kernels (no host round trip).
struct Scalars {
  double* d = nullptr;     // device slots
  double* h = nullptr;     // pinned host mirror
  int cap = 0, top = 0;
  int take(int k) {
    SK_REQUIRE(top + k <= cap, STOKES_ERR_ARG, "scalar slot pool exhausted");
    int s = top;
    top += k;
    return s;
  }
  void give(int k) { top -= k; }
};

// Coefficient read on the device: value = c + s * (*num / *den); null num -> 0
// contribution, null den -> 1. A Krylov coefficient whose denominator must be
// positive (r^T z in a preconditioned CG beta) is built with cg_ratio: a
// denominator <= 0 then sets the context's breakdown flag (bit 1) and the
// coefficient contributes nothing.
struct Coef {
  double c = 0, s = 0;
  const double* num = nullptr;
  const double* den = nullptr;
  int positive = 0;
  static Coef constant(double v) { Coef k; k.c = v; return k; }
  static Coef ratio(const double* num, const double* den, double s = 1.0) {
    Coef k; k.s = s; k.num = num; k.den = den; return k;
  }
  static Coef cg_ratio(const double* num, const double* den, double s = 1.0) {
    Coef k = ratio(num, den, s); k.positive = 1; return k;
  }
};

// ---------------------------------------------------------------------------
// A fixed sequence of multigrid steps (the levels below the finest of one
// V-cycle) executed by one cooperative kernel (mgprog.cu). Step kinds:
// 0 first Chebyshev step from zero (d = y = c1 D^-1 b), 1 y = A x, 2 y += A x,
// 3 y = b - A x, 4 Chebyshev step (d = c1 d + c2 D^-1 (b - A x), y = x + d),
// 5 y = M b with a dense row-major M (m x m). CSR steps have `rows` rows and
// `m` columns; vectors hold nr components (component-major).
// ---------------------------------------------------------------------------
struct MgOp {
  int kind = 0, nr = 1, rows = 0, m = 0;
  const int* rp = nullptr;
  const int* col = nullptr;
  const void* val = nullptr;
  const void* b = nullptr;
  const void* xin = nullptr;
  void* d = nullptr;
  void* y = nullptr;
  const void* dinv = nullptr;
  double c1 = 0, c2 = 0;
};
struct MgOpDev;
// launches a grid barrier that cannot complete; its bounded waits expire and
// set bit 4 of ex.flag (about a second); bar: one device unsigned
void bounded_wait_check(const Exec& ex, unsigned* bar);
struct MgProgram {
  std::vector<MgOp> ops;
  MgOpDev* dev_ops = nullptr;
  unsigned* bar = nullptr;   // grid-barrier counter
  int grid = 0;
  bool f32 = false;
  double bytes = 0;          // algorithmic bytes of one run (sum over steps)
  void* b = nullptr;         // input (right-hand side on the first coarse level)
  void* x = nullptr;         // output (solution on the first coarse level)
  void add(const MgOp& op);
  void finalize(Arena& ar, bool f32);
  void launch(const Exec& ex) const;
};

// ---------------------------------------------------------------------------
// multigrid levels
// ---------------------------------------------------------------------------
struct Level {
  int n = 0;
  int nvi = 0;  // interior P2 nodes (2n-1)^3
  int np = 0;   // P1 nodes (n+1)^3
  double* X = nullptr;  // vertex coordinates of this level
  Csr A3, KQ;           // A~_3 (scalar) and eps M_Q + L_Q
  double *A3_dinv64 = nullptr, *KQ_dinv64 = nullptr;
  float *A3_dinv32 = nullptr, *KQ_dinv32 = nullptr;
  double A3_lmax = 0, KQ_lmax = 0;  // lambda_max(D^{-1} A) estimates
  double* A3_dinv_split64 = nullptr;  // A3 diagonal inverse in parity-split numbering (built on first use)
  float* A3_dinv_split32 = nullptr;
  Csr P2, R2, P1, R1;               // transfers to/from level+1 (P: this <- coarse)
  // coarsest level: dense inverses (row-major)
  double *A3_cinv64 = nullptr, *KQ_cinv64 = nullptr;
  float *A3_cinv32 = nullptr, *KQ_cinv32 = nullptr;
  // 3x3-block velocity preconditioner A~_1 or A~_2 (vel_prec 1, 2): BSR3 on
  // the P2 pattern, point-Jacobi diagonal [3][rows], dense inverse on the
  // coarsest level over the component-major (3 rows) unknowns
  Csr AV;
  double* AV_dinv64 = nullptr;
  float* AV_dinv32 = nullptr;
  double AV_lmax = 0;
  double* AV_cinv64 = nullptr;
  float* AV_cinv32 = nullptr;
};

// ---------------------------------------------------------------------------
// launch wrappers (assembly.cu)
// ---------------------------------------------------------------------------
enum PatternKind { PAT_P2P2 = 0, PAT_P1P1 = 1, PAT_P1P2 = 2, PAT_P2P1 = 3 };
struct StencilTables;  // device stencil offsets
StencilTables* stencils_create(Arena& ar);
void build_pattern(const Exec& ex, Arena& ar, const StencilTables* st, PatternKind kind,
                   int n, Csr& m);

struct AssemblyOut {
  double* a3 = nullptr;     // scalar A~_3 on the P2P2 pattern
  double* abs = nullptr;    // BSR3 A (9 planes) on the P2P2 pattern
  double* mq = nullptr;     // P1 mass on the P1P1 pattern
  double* lq = nullptr;     // P1 Laplacian
  double* kq = nullptr;     // eps M_Q + L_Q
  double* b = nullptr;      // B (3 planes) on the P1P2 pattern
  double* bt = nullptr;     // B^T (3 planes) on the P2P1 pattern
  double* lumped = nullptr; // Lambda_V per interior node
  double* mv = nullptr;     // scalar P2 mass M on the P2P2 pattern
};
// Returns the number of inverted/degenerate tetrahedra.
long long assemble(const Exec& ex, int n, const double* X, double mu, double dt,
                   double eps, const Csr& p2, const Csr& p1, const Csr* b, const Csr* bt,
                   const AssemblyOut& out, int* d_bad);
// |K| per tetrahedron (index 6 * cube + p) of an n^3 Kuhn mesh
void tet_volumes(const Exec& ex, int n, const double* X, double* vol);
// F = M_V f from precomputed tet volumes (vol non-null; else as below)
void assemble_load(const Exec& ex, int n, const double* X, const Csr& p2pat, const double* f_all, double* F,
                   const double* vol);
void assemble_load(const Exec& ex, int n, const double* X, const Csr& p2pat,
                   const double* f_all, double* F);
// out = M_V^T lu on all P2 nodes (lu on interior nodes, 3 components)
void assemble_load_transpose(const Exec& ex, int n, const double* X, const double* lu, double* out);
void build_transfer_p2(const Exec& ex, Arena& ar, int nf, int nc, Csr& P, Csr& R);
void build_transfer_p1(const Exec& ex, Arena& ar, int nf, int nc, Csr& P, Csr& R);
// scalar CSR: dinv[i] = 1 / m_ii; BSR3: dinv[r * rows + i] = 1 / (m_ii)_rr
void diag_inverse(const Exec& ex, const Csr& m, double* dinv);
// out = (1 + g) a_bsr3 - g (a3 on the diagonal of every 3x3 block), same pattern
void combine_grad_div(const Exec& ex, long long nnz, const double* abs, const double* a3, double g, double* out);
// Stencil storage of a square P2-interior (p2 = 1) or P1 (p2 = 0) matrix of
// level size n, values copied from the assembled CSR m (FP64; FP32 on request).
StencilOp* stencil_from_csr(const Exec& ex, Arena& ar, const StencilTables* st, int p2, int n, const Csr& m);
// Symmetric stencil storage of the BSR3 interior-P2 matrix m of level size n
// (FP64 values; FP32 copies are made by the caller).
Sym3Op* sym3_from_csr(const Exec& ex, Arena& ar, const StencilTables* st, int n, const Csr& m);
void to_f32(const Exec& ex, const double* src, float* dst, size_t n);
// lo = FP32(src - hi): with hi = FP32(src), hi + lo carries src to ~2^-48
void to_f32_lo(const Exec& ex, const double* src, const float* hi, float* lo, size_t n);
void subsample_vertices(int nf, int nc, const double* Xf_host, double* Xc_host);

// ---------------------------------------------------------------------------
// sparse products (sparse.cu); T = vector/matrix precision
// ---------------------------------------------------------------------------
// y = A x for a scalar matrix on nr right-hand sides (nr = 1, 3, 4 or 12):
// component-major vectors (component r of row i at r * rows + i), or with il
// node-interleaved ones (at i * nr + r; nr = 4 or 12). The products below
// that take a `split` flag run a stencil-stored P2 matrix with rows and
// columns in parity-split numbering (SplitMap); they require stencil storage
// in use for the given layout (stencil_in_use).
// layout bits of the scalar products: node-interleaved vectors, parity-split
// numbering (both need stencil storage in use for the split)
constexpr int kLayoutIL = 1;
constexpr int kLayoutSplit = 2;
template <class T> void spmv_store(const Exec& ex, const Csr& m, int nr, const T* x, T* y, int kind,
                                   int layout = 0);
// y = b - A x
template <class T> void spmv_resid(const Exec& ex, const Csr& m, int nr, const T* b, const T* x, T* y, int kind,
                                   int layout = 0);
// y += A x
template <class T> void spmv_add(const Exec& ex, const Csr& m, int nr, const T* x, T* y, int kind, int layout = 0);
// Chebyshev step: r = b - A xin; d = c1 d + c2 dinv r; xout = xin + d.
template <class T> void spmv_cheb(const Exec& ex, const Csr& m, int nr, const T* b, const T* xin,
                                  T* d, T* xout, const T* dinv, double c1, double c2, int kind, int layout = 0);
// true if the products of m in this precision and layout read stencil storage
template <class T> bool stencil_in_use(const Csr& m, bool il);
// restriction from a split-numbered fine vector: y = R x with the columns of R
// (natural fine indices) mapped by sm; prolongation into a split-numbered fine
// vector: y += P x with the rows of P mapped by sm
template <class T> void restrict_split(const Exec& ex, const Csr& R, int nr, const T* x, T* y, bool il,
                                      const SplitMap& sm);
template <class T> void prolong_add_split(const Exec& ex, const Csr& P, int nr, const T* x, T* y, bool il,
                                          const SplitMap& sm);
// [nr][rows] (natural) <-> [nr][rows] (split-numbered), or with il the
// interleaved copies to / from split numbering
template <class T> void to_split(const Exec& ex, size_t rows, int nr, const T* src, T* dst, bool il,
                                 const SplitMap& sm);
template <class T> void from_split(const Exec& ex, size_t rows, int nr, const T* src, T* dst, bool il,
                                   const SplitMap& sm);
// the first two Chebyshev steps from x = 0 in one sweep: x1 = d1 = s0 D^-1 b
// formed at each gathered column, then d = c1 d1 + c2 D^-1 (b - A x1),
// xout = x1 + d (il: node-interleaved vectors, nr = 4 or 12)
template <class T> void spmv_cheb_first(const Exec& ex, const Csr& m, int nr, const T* b, T* d, T* xout,
                                        const T* dinv, double s0, double c1, double c2, int kind, int layout = 0);
// BSR3 strain-form A: y = A x or y = b - A x (b may be null).
template <class T> void bsr3_apply(const Exec& ex, const Csr& m, const T* x, T* y, const T* b,
                                   int kind = STOKES_KERNEL_SPMV_A);
// B (1x3 blocks): y = b + alpha B x;  B^T (3x1 blocks): y = b + alpha s o (B^T x),
// s an optional per-row scale (b null: 0). k right-hand sides (1 or 4): x and
// y hold k blocks component-major (velocity [k][3][nvi], pressure [k][np]).
template <class T> void b_apply(const Exec& ex, const Csr& m, const T* x, T* y, const T* b, double alpha,
                                int k = 1);
template <class T> void bt_apply(const Exec& ex, const Csr& m, const T* x, T* y, const T* scale,
                                 const T* b, double alpha, int k = 1);
// y = b - A x for the BSR3 matrix in double-float arithmetic: A = v32 + v32lo,
// x = xh + xl (both FP32 pairs), exact FP32 products (FMA TwoProduct) summed
// with TwoSum; y and b FP64. Relative error ~1e-13 of |A||x| using FP32 units
// only (FP64 throughput is a small fraction of FP32 on this GPU).
void bsr3_residual_df(const Exec& ex, const Csr& m, const float* xh, const float* xl, const double* b, double* y,
                      int kind);
// Chebyshev step on a BSR3 operator with a per-component diagonal dinv[3][rows]
template <class T> void bsr3_cheb(const Exec& ex, const Csr& m, const T* b, const T* xin, T* d, T* xout,
                                  const T* dinv, double c1, double c2, int kind);
template <class T> void dense_apply(const Exec& ex, const T* Minv, int m, int nr, const T* b, T* y,
                                    bool il = false);

// threads per row (m.group, or m.group4 for k = 4 right-hand sides of B / B^T)
void autotune_group(const Exec& ex, Csr& m, int nr, int kind_bsr3, int k = 1);


// ---------------------------------------------------------------------------
// BLAS-1 (blas1.cu). Dot products accumulate in FP64 and reduce in a fixed
// order (deterministic).
// ---------------------------------------------------------------------------
struct DotScratch {
  double* partial = nullptr;   // [kMaxDots][kMaxBlocks]
  unsigned* counter = nullptr;
  // dot products fused into the epilogue of another kernel: one partial per
  // block of that launch (capacity fused_cap), own completion counter
  double* fused_partial = nullptr;
  unsigned* fused_counter = nullptr;
  int fused_cap = 0;
  // dot products of K right-hand sides (multi.cu): partials [K][vectors][blocks]
  // and one completion counter per (right-hand side, vector)
  double* k_partial = nullptr;
  unsigned* k_counter = nullptr;
  long long k_cap = 0;
};

#ifdef __CUDACC__
// Deterministic sum over the grid of one double per thread; every thread of
// every block must call it (no early return before). Warp shuffles, then the
// warps of a block in order, give partial[blockIdx.x]; the last block to
// finish adds the partials in block order, writes *out and resets *counter.
__device__ __forceinline__ void grid_sum(double v, double* partial, unsigned* counter, double* out) {
  __shared__ double sh_[32];
  __shared__ bool last_;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh_[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh_[w];
    partial[blockIdx.x] = t;
    __threadfence();
    last_ = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last_) return;
  __threadfence();
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(&partial[b]);
  for (int o = 16; o; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  __syncthreads();
  if (lane == 0) sh_[wid] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh_[w];
    *out = s;
    *counter = 0u;
  }
}
#endif
constexpr int kMaxDots = 4;
constexpr int kDotBlocks = 608;  // 4 x 152 SMs
// y = A x, and *dot = x . y (deterministic, FP64 accumulation) fused into the
// same kernel when A has symmetric stencil storage (else a separate dot).
template <class T> bool bsr3_apply_dot(const Exec& ex, const Csr& m, const T* x, T* y, const DotScratch& ds,
                                       double* dot);
// symmetric-stencil products (sym3.cu): y = A x or y = b - A x, optional fused
// dot x . (A x); double-float residual y = b - A x
template <class T> void sym3_launch(const Exec& ex, const Csr& m, const T* x, T* y, const T* b, const DotScratch* ds,
                                    double* dot);
// the same (no dot) for four right-hand sides [4][3][rows] in one sweep
template <class T> void sym3_launch4(const Exec& ex, const Csr& m, const T* x, T* y, const T* b);
// k right-hand sides of the BSR3 operator (x, y, b: [k][3][rows]): one sweep
// for k = 4 with symmetric storage, else one product per right-hand side
template <class T> void bsr3_apply_k(const Exec& ex, const Csr& m, int k, const T* x, T* y, const T* b,
                                     int kind = STOKES_KERNEL_SPMV_A);
void sym3_residual_df(const Exec& ex, const Csr& m, const float* xh, const float* xl, const double* b, double* y);
// the same for four right-hand sides [4][3][rows] in one sweep
void sym3_residual_df4(const Exec& ex, const Csr& m, const float* xh, const float* xl, const double* b, double* y);
double sym3_bytes(const Sym3Op& so, int esz, int rows, int streams);
// most blocks of one symmetric-stencil product launch (fused-dot partial capacity)
int sym3_grid(const Sym3Op& so);
// most blocks of one dot-fused BSR3 product launch (fused-dot partial capacity)
int bsr3_dot_grid(const Csr& m);
// FP32 vectors at least this long use compensated FP32 per-thread sums in
// dots() (velocity-sized vectors of the inner solves); shorter ones
// (pressure-sized, the outer Schur iteration) accumulate in FP64 throughout.
constexpr size_t kCompensatedMin = (size_t)1 << 20;
// Stencil storage is used on levels with at least this many rows; smaller
// grids are latency-bound with one thread per row and stay CSR.
constexpr int kStencilMinRows = 1 << 18;
// With several right-hand sides (node-interleaved vectors, 4 or 12 values per
// row) a row carries enough work that the stencil kernel already pays from
// this size on.
constexpr int kStencilMinRowsIL = 1 << 15;
// out[i] = sum_j x_i[j] * y_i[j] for i < k (y_i == nullptr means all ones).
// Accumulation of FP32 dot products: kDotAuto = compensated FP32 partial sums
// for vectors of at least kCompensatedMin entries, kDotFast = compensated for
// any length (inner solves), kDotExact = FP64 throughout (outer Krylov).
enum { kDotAuto = 0, kDotFast = 1, kDotExact = 2 };
template <class T> void dots(const Exec& ex, const DotScratch& ds, int k, const T* const* x,
                             const T* const* y, size_t n, double* out, int mode = kDotAuto);
template <class T> void axpby(const Exec& ex, size_t n, Coef a, const T* x, Coef b, T* y);
// x += a d; r -= a q   (a from device scalars)
template <class T> void cg_update(const Exec& ex, size_t n, Coef a, const T* d, T* x, const T* q, T* r);
// Arnoldi helpers (up to kMaxBasis vectors per call): out[i] = V_i . w (FP64
// accumulation, fixed order, w read once), and w += sign * sum_i h_i V_i with
// h from device scalars (dev_coef) or host constants (host_coef)
constexpr int kMaxBasis = 32;
template <class T> void mdot(const Exec& ex, const DotScratch& ds, int k, const T* const* V, const T* w, size_t n,
                             double* out);
template <class T> void maxpy(const Exec& ex, int k, const double* dev_coef, const double* host_coef, double sign,
                              const T* const* V, T* w, size_t n);
// x += a d; r -= a q; *rr = r . r of the updated r (one kernel)
template <class T> void cg_update_rr(const Exec& ex, const DotScratch& ds, size_t n, Coef a, const T* d, T* x,
                                     const T* q, T* r, double* rr);
// y = a x  (a may be a device ratio)
template <class T> void scale_copy(const Exec& ex, size_t n, Coef a, const T* x, T* y);
// y = c1*x1 + c2*x2 (elementwise, constants)
template <class T> void lincomb2(const Exec& ex, size_t n, double c1, const T* x1, double c2, const T* x2, T* y);
// r -= (*sum / count) (subtract the mean, sum computed beforehand on device)
template <class T> void sub_mean(const Exec& ex, size_t n, const double* sum, double count, T* r);
// x -= (*s1 / *s2) * 1
template <class T> void sub_ratio(const Exec& ex, size_t n, const double* num, const double* den, T* x);
// elementwise y = dinv * x * c (first Chebyshev step from zero: d = x = c D^{-1} b)
template <class T> void cheb_first(const Exec& ex, size_t n, int nr, const T* dinv, const T* b,
                                   double c, T* d, T* x);
// the same on node-interleaved vectors (row i's nr values at i * nr)
template <class T> void cheb_first_il(const Exec& ex, size_t n, int nr, const T* dinv, const T* b, double c, T* d,
                                      T* x);
// component-major [nr][rows] <-> node-interleaved [rows][nr] (nr = 4 or 12)
template <class T> void to_interleaved(const Exec& ex, size_t rows, int nr, const T* cm, T* il);
template <class T> void to_component_major(const Exec& ex, size_t rows, int nr, const T* il, T* cm);
template <class S, class D> void convert(const Exec& ex, size_t n, const S* x, D* y);
// hi = FP32(x), lo = FP32(x - hi)
void split_f64(const Exec& ex, size_t n, const double* x, float* hi, float* lo);
template <class S, class D> void add_convert(const Exec& ex, size_t n, const S* x, D* y);

// ---------------------------------------------------------------------------
// K right-hand sides in lockstep (multi.cu). A K-vector stores K systems'
// reduced unknowns as the velocity blocks [K][nu] followed by the pressure
// blocks [K][np]; `parts` selects the velocity (1), pressure (2) or both (3)
// parts of each right-hand side's segment. Vectors of K plain blocks of
// length n are K-vectors with nu = n, np = 0, parts = 1.
// ---------------------------------------------------------------------------
constexpr int kMaxRhs = 8;
constexpr int kMaxBasisK = 32;
// Per-right-hand-side coefficient: value(k) = c[k] + s * num[k*stride] /
// den[k*stride] (device scalars; null num: c[k] alone), 0 for a right-hand
// side whose bit in `active` is clear. `positive`: as Coef::cg_ratio.
struct KCoefs {
  double c[kMaxRhs] = {};
  double s = 0;
  const double* num = nullptr;
  const double* den = nullptr;
  int stride = 1;
  int positive = 0;
  unsigned active = ~0u;
  static KCoefs constant(double v) {
    KCoefs k;
    for (int i = 0; i < kMaxRhs; ++i) k.c[i] = v;
    return k;
  }
  static KCoefs host(const double* v, int K) {
    KCoefs k;
    for (int i = 0; i < K; ++i) k.c[i] = v[i];
    return k;
  }
  static KCoefs ratio(const double* num, const double* den, double s = 1.0, int stride = 1) {
    KCoefs k;
    k.s = s;
    k.num = num;
    k.den = den;
    k.stride = stride;
    return k;
  }
  static KCoefs cg_ratio(const double* num, const double* den, double s = 1.0, int stride = 1) {
    KCoefs k = ratio(num, den, s, stride);
    k.positive = 1;
    return k;
  }
  KCoefs& mask(unsigned m) {
    active = m;
    return *this;
  }
#ifdef __CUDACC__
  __device__ double value(int k, int* flag) const {
    if (!((active >> k) & 1u)) return 0.0;
    double v = c[k];
    if (num) {
      const double dn = den ? den[(size_t)k * stride] : 1.0;
      if (positive && !(dn > 0.0)) {
        if (flag) atomicOr(flag, 1);
        return v;
      }
      if (dn != 0.0) v += s * num[(size_t)k * stride] / dn;
    }
    return v;
  }
#endif
};
template <class T> struct KBasis {
  const T* v[kMaxBasisK];
};
struct KHost {
  double c[kMaxRhs * kMaxBasisK];
};
// out[k] = x_k . y_k over the segment (y null: sum of x_k), FP64 accumulation
template <class T> void kdot(const Exec& ex, const DotScratch& ds, size_t nu, size_t np, int K, int parts, const T* x,
                             const T* y, double* out);
// y_k = a_k x_k + b_k y_k over the segment
template <class T> void kaxpby(const Exec& ex, size_t nu, size_t np, int K, int parts, const KCoefs& a, const T* x,
                               const KCoefs& b, T* y);
// y_k += c_k over the segment
template <class T> void kaddconst(const Exec& ex, size_t nu, size_t np, int K, int parts, const KCoefs& c, T* y);
// Arnoldi helpers over whole segments (parts = 3) of J <= kMaxBasisK
// K-vectors: out[k * ld + i] = V_i(k) . w(k); w(k) += sign * sum_i h_ki V_i(k)
// with h_ki = h[k * ld + i] (device) or hhost[k * ld + i] (host)
template <class T> void kmdot(const Exec& ex, const DotScratch& ds, size_t nu, size_t np, int K, int J,
                              const T* const* V, const T* w, double* out, int ld);
template <class T> void kmaxpy(const Exec& ex, size_t nu, size_t np, int K, int J, const T* const* V, const double* h,
                               const double* hhost, int ld, double sign, T* w);
// out[k] = a[k] - b[k] for k < K (device scalars)
void ksub(const Exec& ex, int K, double* out, const double* a, const double* b);
// scratch doubles the K-dot kernels need (capacity of DotScratch::k_partial)
long long kdot_scratch(size_t len_max, int K);
void expand_velocity(const Exec& ex, int n, const double* ured, double* uall);
void restrict_velocity(const Exec& ex, int n, const double* uall, double* ured);
void count_nonfinite(const Exec& ex, size_t n, const double* x, int* flag);

}  // namespace sk

// ---------------------------------------------------------------------------
// the context (defined in capi.cu, used by solver.cu)
// ---------------------------------------------------------------------------
struct stokes_ctx {
  int n = 0;
  double mu = 0, dt = 0, gamma = 0;
  stokes_options opt{};
  sk::Exec ex;
  sk::Prof prof;
  sk::Arena arena;
  sk::VecPool pool;
  sk::Scalars sc;
  sk::DotScratch ds;
  int* d_flag = nullptr;
  std::vector<sk::Level> lv;
  sk::Csr A, B, Bt, MQ, LQ;  // fine level (P2P2 BSR3, P1P2, P2P1, P1P1, P1P1)
  double* lumped = nullptr;  // Lambda_V per interior node
  double* tet_vol = nullptr; // |K| of every tetrahedron of the finest mesh (6 per cube)
  sk::Csr MV;                // scalar P2 mass (C_lambda only); M_V = MV per component
  double* MV_dinv64 = nullptr;
  float* MV_dinv32 = nullptr;
  double *lumped_inv64 = nullptr;
  float* lumped_inv32 = nullptr;
  double* MQ_dinv64 = nullptr;
  float* MQ_dinv32 = nullptr;
  double* MQ1 = nullptr;     // M_Q 1
  double MQ1_sum = 0;
  bool mixed = false;
  // last forward solution (reduced) for the adjoint
  std::vector<std::unique_ptr<sk::StencilOp>> stencils;  // owned stencil storages
  std::unique_ptr<sk::Sym3Op> symA;                       // A in symmetric stencil storage
  double* U_last = nullptr;
  double* P_last = nullptr;
  bool have_solution = false;
  // host staging for *_host calls
  double *f_dev = nullptr, *g_dev = nullptr, *u_dev = nullptr, *p_dev = nullptr;
  cudaEvent_t ev_read = nullptr;  // host reads of device scalars
  cudaEvent_t ev_sync = nullptr;  // host waits for the stream (blocking-sync with host_wait = 1)
  // levels >= 1 of the V-cycle of A~_3 (which = 0), of eps M_Q + L_Q
  // (which = 1) and of the block operator A~_1 / A~_2 (which = 2), FP64 [0]
  // and FP32 [1]: fixed input/output vectors, a private
  // vector pool for the temporaries, and the captured graph
  struct CoarseGraph {
    int state = 0;  // 0: next call runs eagerly, 1: next call captures, 2: replay
    void* b = nullptr;
    void* x = nullptr;
    sk::VecPool pool;
    cudaGraphExec_t exec = nullptr;
    sk::Prof::Counts counts;
  } cgraph[3][2];
  // levels >= 1 of a V-cycle (which = 0, 1) in one cooperative kernel, FP64 [0]
  // and FP32 [1] (built on first use)
  std::unique_ptr<sk::MgProgram> mgprog[2][2];
  // graphs are captured on this private stream (capture is not allowed on the
  // legacy default stream) and launched on ex.s
  cudaStream_t cap_stream = nullptr;
  // whole V-cycles (all levels) replayed from graphs, keyed by (which, FP32,
  // b, x, cycles): the vector pool hands the same buffers to the same call
  // site, so a few keys recur. One private pool serves all of them (they run
  // one at a time on ex.s). in_cycle_graph: a whole-cycle graph is being
  // recorded or warmed, so nested V-cycle levels run as plain launches.
  struct CycleGraph {
    int seen = 0;
    cudaGraphExec_t exec = nullptr;
    sk::Prof::Counts counts;
  };
  std::map<std::tuple<int, int, const void*, void*, int>, CycleGraph> vgraphs;
  sk::VecPool vgraph_pool;
  bool in_cycle_graph = false;
  bool graphs_off = false;  // a region could not be recorded: plain launches from then on
  double setup_ms[STOKES_SETUP_PHASES] = {};  // wall-clock ms per setup phase
  // counters
  int outer_iters = 0, inner_iters = 0, schur_inner_iters = 0;
  bool outer_capped = false, inner_capped = false;
};

namespace sk {
void setup_context(stokes_ctx* c, int n, const double* Xhost);
int solve_multi_context(stokes_ctx* c, int k, const double* f, const double* g, double tol, double* u,
                        double* p, stokes_info* info);
int solve_context(stokes_ctx* c, const double* f, const double* g, double tol, double* u,
                  double* p, stokes_info* info);
int adjoint_context(stokes_ctx* c, const double* dJdu, const double* dJdp, double tol,
                    double* dJdf, double* dJdg, double* dJdmu, stokes_info* info);
void apply_operator(stokes_ctx* c, int op, int level, const double* x, double* y);
double estimate_lmax(stokes_ctx& c, const Csr& M, const double* dinv, int steps, uint64_t seed);
// velocity V-cycle kind: 0 (scalar A~_3 per component) or 2 (block A~_1 / A~_2)
inline int velocity_cycle(const stokes_ctx& c) { return c.opt.vel_prec == 3 ? 0 : 2; }
void set_last_error(const std::string& msg);  // message returned by stokes_last_error()
void scalar_sub(const Exec& ex, double* out, const double* a, const double* b);
}  // namespace sk
