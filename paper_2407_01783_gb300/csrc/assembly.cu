// Mesh-structured sparsity patterns, element-coloured FEM assembly, load
// vectors and multigrid transfer operators for P2-P1 on Kuhn meshes.
//
// Matrices follow the paper's definitions (Sec. 2.2 "Discrete problem"):
//   M_V,ij = int phi_i . phi_j,  E_V = int 2 eps(phi_i):eps(phi_j),
//   A = M_V/dt + mu E_V,  B_kj = int psi_k div phi_j,
// Sec. 3.2 (L_V, Eq. precond_A_plus_lambda_D_3: A~_3 = M_V/dt + mu L_V) and
// Sec. 4.1-4.2 (M_Q, L_Q, eps M_Q + L_Q, lumped Lambda_V,ii = int |phi_i|).
// Homogeneous Dirichlet velocity (Sec. 3.1): only interior P2 nodes carry
// velocity unknowns. Element integrals use the 4-point degree-2 rule on each
// affine tetrahedron (exact for products of two P2 gradients and for
// P1 x P2-gradient), and the closed-form P2 mass matrix (entries / 420).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

#include "internal.h"

namespace sk {

// ---------------------------------------------------------------------------
// Kuhn reference cube: six tets, tet p has vertices 0, e_p0, e_p0 + e_p1, 1.
// ---------------------------------------------------------------------------
static const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
static const int kPermSign[6] = {+1, -1, -1, +1, +1, -1};
static const int kEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

__constant__ int c_perm[6][3];
__constant__ int c_perm_sign[6];
__constant__ int c_edge[6][2];

static void upload_constants() {
  SK_CUDA(cudaMemcpyToSymbol(c_perm, kPerm, sizeof(kPerm)));
  SK_CUDA(cudaMemcpyToSymbol(c_perm_sign, kPermSign, sizeof(kPermSign)));
  SK_CUDA(cudaMemcpyToSymbol(c_edge, kEdge, sizeof(kEdge)));
}

static void ref_tet(int p, int v[4][3]) {
  for (int c = 0; c < 3; ++c) v[0][c] = 0, v[3][c] = 1;
  for (int c = 0; c < 3; ++c) v[1][c] = (c == kPerm[p][0]);
  for (int c = 0; c < 3; ++c) v[2][c] = v[1][c] + (c == kPerm[p][1]);
}

// ---------------------------------------------------------------------------
// stencils: for each row class (parity of the half-grid coordinates) the
// half-grid offsets of every node sharing a tetrahedron with the row node.
// Every tet is an even translate of one reference-cube tet, so scanning the
// reference cube gives the complete sets.
// ---------------------------------------------------------------------------
struct StencilTables {
  int* d_off = nullptr;       // 3 ints per offset
  int beg[4][9];              // per pattern kind: offsets of class c in [beg[c], beg[c+1])
  std::vector<int> h_off;     // host copy of the offsets
};

StencilTables* stencils_create(Arena& ar) {
  using Off = std::array<int, 3>;
  auto key = [](const Off& o) { return std::make_tuple(o[2], o[1], o[0]); };
  auto cmp = [&](const Off& a, const Off& b) { return key(a) < key(b); };
  std::vector<std::set<Off, decltype(cmp)>> sets;
  for (int k = 0; k < 4 * 8; ++k) sets.emplace_back(cmp);
  for (int p = 0; p < 6; ++p) {
    int v[4][3];
    ref_tet(p, v);
    int q[10][3];
    for (int l = 0; l < 4; ++l)
      for (int c = 0; c < 3; ++c) q[l][c] = 2 * v[l][c];
    for (int e = 0; e < 6; ++e)
      for (int c = 0; c < 3; ++c) q[4 + e][c] = v[kEdge[e][0]][c] + v[kEdge[e][1]][c];
    auto cls = [](const int* x) { return (x[0] & 1) | ((x[1] & 1) << 1) | ((x[2] & 1) << 2); };
    for (int a = 0; a < 10; ++a) {
      for (int b = 0; b < 10; ++b)
        sets[PAT_P2P2 * 8 + cls(q[a])].insert({q[b][0] - q[a][0], q[b][1] - q[a][1], q[b][2] - q[a][2]});
      for (int l = 0; l < 4; ++l)
        sets[PAT_P2P1 * 8 + cls(q[a])].insert({q[l][0] - q[a][0], q[l][1] - q[a][1], q[l][2] - q[a][2]});
    }
    for (int l = 0; l < 4; ++l) {
      for (int m = 0; m < 4; ++m)
        sets[PAT_P1P1 * 8].insert({q[m][0] - q[l][0], q[m][1] - q[l][1], q[m][2] - q[l][2]});
      for (int b = 0; b < 10; ++b)
        sets[PAT_P1P2 * 8].insert({q[b][0] - q[l][0], q[b][1] - q[l][1], q[b][2] - q[l][2]});
    }
  }
  std::vector<int> flat;
  auto* st = new StencilTables();
  for (int kind = 0; kind < 4; ++kind)
    for (int c = 0; c < 8; ++c) {
      st->beg[kind][c] = (int)(flat.size() / 3);
      for (const Off& o : sets[kind * 8 + c]) flat.insert(flat.end(), o.begin(), o.end());
      st->beg[kind][c + 1] = (int)(flat.size() / 3);
    }
  st->h_off = flat;
  st->d_off = ar.alloc<int>(flat.size());
  SK_CUDA(cudaMemcpy(st->d_off, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice));
  upload_constants();
  return st;
}

// Index spaces on the half-grid: q = lo + step * i, 0 <= i < ext per axis.
struct Space {
  int lo, step, ext;
};
__host__ __device__ inline Space p2_interior_space(int n) { return Space{1, 1, 2 * n - 1}; }
__host__ __device__ inline Space p1_space(int n) { return Space{0, 2, n + 1}; }

__device__ __forceinline__ int space_index(const Space& s, int q) {
  int t = q - s.lo;
  if (t < 0) return -1;
  if (s.step == 2) {
    if (t & 1) return -1;
    t >>= 1;
  }
  return t < s.ext ? t : -1;
}

struct Beg9 {
  int b[9];
};

__global__ void k_pattern(int pass, int rows, Space rs, Space cs, const int* __restrict__ off,
                          Beg9 beg, int* __restrict__ cnt_or_rowptr, int* __restrict__ col) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  int e = rs.ext;
  int q0 = rs.lo + rs.step * (r % e);
  int q1 = rs.lo + rs.step * ((r / e) % e);
  int q2 = rs.lo + rs.step * (r / (e * e));
  int cls = (q0 & 1) | ((q1 & 1) << 1) | ((q2 & 1) << 2);
  int w = pass ? cnt_or_rowptr[r] : 0;
  int count = 0;
  for (int k = beg.b[cls]; k < beg.b[cls + 1]; ++k) {
    int c0 = space_index(cs, q0 + off[3 * k]);
    int c1 = space_index(cs, q1 + off[3 * k + 1]);
    int c2 = space_index(cs, q2 + off[3 * k + 2]);
    if (c0 < 0 || c1 < 0 || c2 < 0) continue;
    if (pass)
      col[w++] = c0 + cs.ext * (c1 + cs.ext * c2);
    else
      ++count;
  }
  if (!pass) cnt_or_rowptr[r] = count;
}

// exclusive scan of counts[0..rows) into rowptr[0..rows] (block sums on host)
__global__ void k_block_sum(const int* __restrict__ cnt, int rows, long long* __restrict__ bsum) {
  __shared__ long long sh[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long v = i < rows ? cnt[i] : 0;
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = v;
  }
}

__global__ void k_block_scan(const int* __restrict__ cnt, int rows, const long long* __restrict__ boff,
                             int* __restrict__ rowptr) {
  __shared__ long long sh[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long v = i < rows ? cnt[i] : 0;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    sh[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  long long before = (wid ? sh[wid - 1] : 0) + incl - v;
  if (i < rows) rowptr[i] = (int)(boff[blockIdx.x] + before);
}

static void scan_counts(const Exec& ex, Arena& ar, const int* cnt, int rows, int* rowptr, long long* total) {
  const int bs = 1024;
  int nb = cdiv(rows, bs);
  long long* bsum = nullptr;
  SK_CUDA(cudaMalloc(&bsum, sizeof(long long) * nb));
  k_block_sum<<<nb, bs, 0, ex.s>>>(cnt, rows, bsum);
  SK_CHECK_LAUNCH();
  std::vector<long long> h(nb);
  SK_CUDA(cudaMemcpyAsync(h.data(), bsum, sizeof(long long) * nb, cudaMemcpyDeviceToHost, ex.s));
  SK_CUDA(cudaStreamSynchronize(ex.s));
  long long run = 0;
  for (int b = 0; b < nb; ++b) {
    long long t = h[b];
    h[b] = run;
    run += t;
  }
  SK_REQUIRE(run < (1LL << 31), STOKES_ERR_ARG, "sparse pattern exceeds 2^31 entries");
  SK_CUDA(cudaMemcpyAsync(bsum, h.data(), sizeof(long long) * nb, cudaMemcpyHostToDevice, ex.s));
  k_block_scan<<<nb, bs, 0, ex.s>>>(cnt, rows, bsum, rowptr);
  SK_CHECK_LAUNCH();
  int tot = (int)run;
  SK_CUDA(cudaMemcpyAsync(rowptr + rows, &tot, sizeof(int), cudaMemcpyHostToDevice, ex.s));
  SK_CUDA(cudaStreamSynchronize(ex.s));
  SK_CUDA(cudaFree(bsum));
  (void)ar;
  *total = run;
}

void build_pattern(const Exec& ex, Arena& ar, const StencilTables* st, PatternKind kind, int n, Csr& m) {
  Space rs = (kind == PAT_P2P2 || kind == PAT_P2P1) ? p2_interior_space(n) : p1_space(n);
  Space cs = (kind == PAT_P2P2 || kind == PAT_P1P2) ? p2_interior_space(n) : p1_space(n);
  long long rows = (long long)rs.ext * rs.ext * rs.ext;
  long long cols = (long long)cs.ext * cs.ext * cs.ext;
  m.rows = (int)rows;
  m.cols = (int)cols;
  m.rowptr = ar.alloc<int>(rows + 1);
  Beg9 beg;
  for (int c = 0; c < 9; ++c) beg.b[c] = st->beg[kind][c];
  int bs = 256, nb = cdiv(rows, bs);
  k_pattern<<<nb, bs, 0, ex.s>>>(0, m.rows, rs, cs, st->d_off, beg, m.rowptr, nullptr);
  SK_CHECK_LAUNCH();
  long long total = 0;
  int* cnt = ar.alloc<int>(rows);
  SK_CUDA(cudaMemcpyAsync(cnt, m.rowptr, sizeof(int) * rows, cudaMemcpyDeviceToDevice, ex.s));
  scan_counts(ex, ar, cnt, m.rows, m.rowptr, &total);
  m.nnz = total;
  m.col = ar.alloc<int>(total);
  k_pattern<<<nb, bs, 0, ex.s>>>(1, m.rows, rs, cs, st->d_off, beg, m.rowptr, m.col);
  SK_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// element-coloured assembly
// ---------------------------------------------------------------------------
// Closed-form P2 mass matrix on a tetrahedron, times 420/|K|: vertex-vertex 6
// (diagonal) or 1; vertex-edge -4 if the vertex is an end of the edge, else
// -6; edge-edge 32 (diagonal), 16 if the edges share a vertex, else 8.
__device__ __forceinline__ double p2_mass420(int a, int b) {
  if (a < 4 && b < 4) return a == b ? 6.0 : 1.0;
  if (a >= 4 && b >= 4) {
    if (a == b) return 32.0;
    int e = a - 4, f = b - 4;
    bool share = c_edge[e][0] == c_edge[f][0] || c_edge[e][0] == c_edge[f][1] ||
                 c_edge[e][1] == c_edge[f][0] || c_edge[e][1] == c_edge[f][1];
    return share ? 16.0 : 8.0;
  }
  int v = a < 4 ? a : b, e = (a < 4 ? b : a) - 4;
  return (c_edge[e][0] == v || c_edge[e][1] == v) ? -4.0 : -6.0;
}

// position of column c in col[lo, hi) (sorted), or -1 if absent
__device__ __forceinline__ int find_col(const int* __restrict__ col, int lo, int hi, int c) {
  int end = hi;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (col[mid] < c) lo = mid + 1; else hi = mid;
  }
  return (lo < end && col[lo] == c) ? lo : -1;
}

struct TetGeom {
  double g[4][3];  // barycentric gradients
  double vol;
  int v[4][3];     // integer vertex coordinates
  bool ok;
};

__device__ inline void tet_geometry(int n, const double* __restrict__ X, int i, int j, int k, int p, TetGeom& t) {
  const int nv = n + 1;
  for (int c = 0; c < 3; ++c) {
    t.v[0][c] = (c == 0 ? i : c == 1 ? j : k);
    t.v[3][c] = t.v[0][c] + 1;
    t.v[1][c] = t.v[0][c] + (c == c_perm[p][0]);
    t.v[2][c] = t.v[1][c] + (c == c_perm[p][1]);
  }
  double x[4][3];
  for (int l = 0; l < 4; ++l) {
    size_t id = (size_t)t.v[l][0] + nv * ((size_t)t.v[l][1] + (size_t)nv * t.v[l][2]);
    for (int c = 0; c < 3; ++c) x[l][c] = X[3 * id + c];
  }
  double e1[3], e2[3], e3[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = x[1][c] - x[0][c];
    e2[c] = x[2][c] - x[0][c];
    e3[c] = x[3][c] - x[0][c];
  }
  double c23[3] = {e2[1] * e3[2] - e2[2] * e3[1], e2[2] * e3[0] - e2[0] * e3[2], e2[0] * e3[1] - e2[1] * e3[0]};
  double c31[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
  double c12[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double det = e1[0] * c23[0] + e1[1] * c23[1] + e1[2] * c23[2];
  t.ok = isfinite(det) && det * c_perm_sign[p] > 0.0;
  double inv = 1.0 / det;
  for (int c = 0; c < 3; ++c) {
    t.g[1][c] = c23[c] * inv;  // rows of J^{-1}, J = [e1 e2 e3]
    t.g[2][c] = c31[c] * inv;
    t.g[3][c] = c12[c] * inv;
    t.g[0][c] = -(t.g[1][c] + t.g[2][c] + t.g[3][c]);
  }
  t.vol = fabs(det) / 6.0;
}

// half-grid coordinates of local node a (vertices 0..3, edges 4..9)
__device__ __forceinline__ void local_node(const TetGeom& t, int a, int q[3]) {
  if (a < 4) {
    for (int c = 0; c < 3; ++c) q[c] = 2 * t.v[a][c];
  } else {
    int l = c_edge[a - 4][0], m = c_edge[a - 4][1];
    for (int c = 0; c < 3; ++c) q[c] = t.v[l][c] + t.v[m][c];
  }
}

__device__ __forceinline__ int p2_interior_index(int n, const int q[3]) {
  int m = 2 * n - 1;
  if (q[0] < 1 || q[0] > m || q[1] < 1 || q[1] > m || q[2] < 1 || q[2] > m) return -1;
  return (q[0] - 1) + m * ((q[1] - 1) + m * (q[2] - 1));
}

// degree-2 rule: lam = alpha at one vertex, beta at the others, weight |K|/4
#define QA 0.5854101966249685
#define QB 0.1381966011250105

// gradient of the P2 basis function a at quadrature point qp
__device__ __forceinline__ void p2_grad(const TetGeom& t, int a, int qp, double g[3]) {
  if (a < 4) {
    double lam = qp == a ? QA : QB;
    double s = 4.0 * lam - 1.0;
    for (int c = 0; c < 3; ++c) g[c] = s * t.g[a][c];
  } else {
    int l = c_edge[a - 4][0], m = c_edge[a - 4][1];
    double ll = qp == l ? QA : QB, lm = qp == m ? QA : QB;
    for (int c = 0; c < 3; ++c) g[c] = 4.0 * (ll * t.g[m][c] + lm * t.g[l][c]);
  }
}

struct AsmArgs {
  int n;
  const double* X;
  double mu, dt, eps;
  int cx, cy, cz, mx, my, mz;
  const int *p2rp, *p2col;
  long long p2nnz;
  const int *p1rp, *p1col;
  long long p1nnz;
  const int *brp, *bcol;
  long long bnnz;
  const int *btrp, *btcol;
  long long btnnz;
  AssemblyOut o;
  int* bad;
  int p;  // tetrahedron of the cube handled by this launch
};

// One launch per (colour, tetrahedron p of the cube) and one thread per (cube
// of the colour, local node ra of tet p): the thread adds tet p's
// contributions to velocity row ra (and, for a vertex, to pressure row ra).
// Cubes of one colour share no node and the ten local nodes of one tet are
// distinct, so no two threads of a launch write the same entry; launching the
// colours and then the six tets in order keeps the summation order of every
// entry fixed (deterministic assembly).
__global__ void __launch_bounds__(128) k_assemble(AsmArgs a) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.mx * a.my * a.mz * 10) return;
  const int ra = t % 10;
  t /= 10;
  int i = 2 * (t % a.mx) + a.cx;
  int j = 2 * ((t / a.mx) % a.my) + a.cy;
  int k = 2 * (t / (a.mx * a.my)) + a.cz;
  const int n = a.n, nv = n + 1;
  const int p = a.p;
  {
    TetGeom tg;
    tet_geometry(n, a.X, i, j, k, p, tg);
    if (!tg.ok) {
      if (ra == 0) atomicAdd(a.bad, 1);
      return;
    }
    const double w = tg.vol * 0.25;
    int ri[10];
    for (int l = 0; l < 10; ++l) {
      int q[3];
      local_node(tg, l, q);
      ri[l] = p2_interior_index(n, q);
    }
    int vid[4];
    for (int l = 0; l < 4; ++l) vid[l] = tg.v[l][0] + nv * (tg.v[l][1] + nv * tg.v[l][2]);
    double gq[4][10][3];
    for (int qp = 0; qp < 4; ++qp)
      for (int l = 0; l < 10; ++l) p2_grad(tg, l, qp, gq[qp][l]);
    // velocity row ra
    {
      int row = ri[ra];
      if (row >= 0) {
      if (a.o.lumped) a.o.lumped[row] += tg.vol * (ra < 4 ? 3.0 / 32.0 : 1.0 / 5.0);
      if (a.o.a3 || a.o.abs || a.o.mv) {
        int lo = a.p2rp[row], hi = a.p2rp[row + 1];
        for (int cb = 0; cb < 10; ++cb) {
          int colj = ri[cb];
          if (colj < 0) continue;
          double G[3][3];
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) {
              double s = 0;
              for (int qp = 0; qp < 4; ++qp) s += gq[qp][ra][c] * gq[qp][cb][d];
              G[c][d] = w * s;
            }
          double mass = tg.vol * p2_mass420(ra, cb) / 420.0;
          double lap = G[0][0] + G[1][1] + G[2][2];
          double diag = mass / a.dt + a.mu * lap;
          int pos = find_col(a.p2col, lo, hi, colj);
          if (pos < 0) {
            atomicAdd(a.bad, 1);
            continue;
          }
          if (a.o.a3) a.o.a3[pos] += diag;
          if (a.o.mv) a.o.mv[pos] += mass;
          if (a.o.abs) {
            // 2 eps(phi_a e_c):eps(phi_b e_d) = delta_cd grad.grad + d_d phi_a d_c phi_b
            for (int c = 0; c < 3; ++c)
              for (int d = 0; d < 3; ++d)
                a.o.abs[(size_t)(c * 3 + d) * a.p2nnz + pos] += (c == d ? diag : 0.0) + a.mu * G[d][c];
          }
        }
      }
      if (a.o.bt) {
        int lo = a.btrp[row], hi = a.btrp[row + 1];
        for (int l = 0; l < 4; ++l) {
          int pos = find_col(a.btcol, lo, hi, vid[l]);
          if (pos < 0) {
            atomicAdd(a.bad, 1);
            continue;
          }
          for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int qp = 0; qp < 4; ++qp) s += (qp == l ? QA : QB) * gq[qp][ra][c];
            a.o.bt[(size_t)c * a.btnnz + pos] += w * s;
          }
        }
      }
      }
    }
    // pressure row of vertex ra
    if (ra < 4) {
      const int l = ra;
      int row = vid[l];
      if (a.o.mq || a.o.lq || a.o.kq) {
        int lo = a.p1rp[row], hi = a.p1rp[row + 1];
        for (int m = 0; m < 4; ++m) {
          int pos = find_col(a.p1col, lo, hi, vid[m]);
          if (pos < 0) {
            atomicAdd(a.bad, 1);
            continue;
          }
          double mm = tg.vol * (l == m ? 2.0 : 1.0) / 20.0;
          double ll = tg.vol * (tg.g[l][0] * tg.g[m][0] + tg.g[l][1] * tg.g[m][1] + tg.g[l][2] * tg.g[m][2]);
          if (a.o.mq) a.o.mq[pos] += mm;
          if (a.o.lq) a.o.lq[pos] += ll;
          if (a.o.kq) a.o.kq[pos] += a.eps * mm + ll;
        }
      }
      if (a.o.b) {
        int lo = a.brp[row], hi = a.brp[row + 1];
        for (int cb = 0; cb < 10; ++cb) {
          int colj = ri[cb];
          if (colj < 0) continue;
          int pos = find_col(a.bcol, lo, hi, colj);
          if (pos < 0) {
            atomicAdd(a.bad, 1);
            continue;
          }
          for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int qp = 0; qp < 4; ++qp) s += (qp == l ? QA : QB) * gq[qp][cb][c];
            a.o.b[(size_t)c * a.bnnz + pos] += w * s;
          }
        }
      }
    }
  }
}

long long assemble(const Exec& ex, int n, const double* X, double mu, double dt, double eps,
                   const Csr& p2, const Csr& p1, const Csr* b, const Csr* bt, const AssemblyOut& out,
                   int* d_bad) {
  auto zero = [&](double* p, size_t cnt) {
    if (p) SK_CUDA(cudaMemsetAsync(p, 0, cnt * sizeof(double), ex.s));
  };
  zero(out.a3, p2.nnz);
  zero(out.mv, p2.nnz);
  zero(out.abs, 9 * (size_t)p2.nnz);
  zero(out.mq, p1.nnz);
  zero(out.lq, p1.nnz);
  zero(out.kq, p1.nnz);
  if (b) zero(out.b, 3 * (size_t)b->nnz);
  if (bt) zero(out.bt, 3 * (size_t)bt->nnz);
  zero(out.lumped, p2.rows);
  SK_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), ex.s));
  AsmArgs a{};
  a.n = n;
  a.X = X;
  a.mu = mu;
  a.dt = dt;
  a.eps = eps;
  a.p2rp = p2.rowptr;
  a.p2col = p2.col;
  a.p2nnz = p2.nnz;
  a.p1rp = p1.rowptr;
  a.p1col = p1.col;
  a.p1nnz = p1.nnz;
  if (b) a.brp = b->rowptr, a.bcol = b->col, a.bnnz = b->nnz;
  if (bt) a.btrp = bt->rowptr, a.btcol = bt->col, a.btnnz = bt->nnz;
  a.o = out;
  a.bad = d_bad;
  // colour = parity of the cube index: cubes of one colour share no node.
  for (int colour = 0; colour < 8; ++colour) {
    a.cx = colour & 1;
    a.cy = (colour >> 1) & 1;
    a.cz = (colour >> 2) & 1;
    a.mx = (n - a.cx + 1) / 2;
    a.my = (n - a.cy + 1) / 2;
    a.mz = (n - a.cz + 1) / 2;
    int cubes = a.mx * a.my * a.mz;
    if (cubes == 0) continue;
    for (int p = 0; p < 6; ++p) {
      a.p = p;
      k_assemble<<<cdiv((long long)cubes * 10, 128), 128, 0, ex.s>>>(a);
      SK_CHECK_LAUNCH();
    }
  }
  int bad = 0;
  SK_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, ex.s));
  SK_CUDA(cudaStreamSynchronize(ex.s));
  return bad;
}

// F = M_V f_h on interior rows (f_h: P2 interpolant of the nodal force at all nodes)
struct LoadArgs {
  int n;
  const double* X;
  int cx, cy, cz, mx, my, mz;
  const double* f;
  double* F;
  int p;  // tetrahedron of the cube handled by this launch (k_load)
};

// One launch per (colour, tet p), one thread per (cube, local node ra): the
// same ownership argument and summation order as k_assemble.
__global__ void __launch_bounds__(128) k_load(LoadArgs a) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.mx * a.my * a.mz * 10) return;
  const int ra = t % 10;
  t /= 10;
  int i = 2 * (t % a.mx) + a.cx;
  int j = 2 * ((t / a.mx) % a.my) + a.cy;
  int k = 2 * (t / (a.mx * a.my)) + a.cz;
  const int N = 2 * a.n + 1;
  TetGeom tg;
  tet_geometry(a.n, a.X, i, j, k, a.p, tg);
  if (!tg.ok) return;
  int q[3];
  local_node(tg, ra, q);
  const int row = p2_interior_index(a.n, q);
  if (row < 0) return;
  double s[3] = {0, 0, 0};
  for (int cb = 0; cb < 10; ++cb) {
    local_node(tg, cb, q);
    const size_t gid = (size_t)q[0] + N * ((size_t)q[1] + (size_t)N * q[2]);
    const double m = p2_mass420(ra, cb);
    for (int c = 0; c < 3; ++c) s[c] += m * a.f[3 * gid + c];
  }
  const size_t nvi = (size_t)(2 * a.n - 1) * (2 * a.n - 1) * (2 * a.n - 1);
  for (int c = 0; c < 3; ++c) a.F[c * nvi + row] += tg.vol * s[c] / 420.0;  // component-major
}

// |K| of every tetrahedron, index 6 * cube + p (cube lexicographic, x fastest)
__global__ void k_tet_volumes(int n, const double* __restrict__ X, double* __restrict__ vol) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6LL * n * n * n) return;
  const int p = (int)(t % 6);
  const long long cube = t / 6;
  const int i = (int)(cube % n), j = (int)((cube / n) % n), k = (int)(cube / ((long long)n * n));
  TetGeom tg;
  tet_geometry(n, X, i, j, k, p, tg);
  vol[t] = tg.vol;
}

static void upload_tet_nodes();
void tet_volumes(const Exec& ex, int n, const double* X, double* vol) {
  {  // the node table of the load kernel, once per device (setup runs before any solve)
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    SK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && !done[dev]) {
      upload_tet_nodes();
      done[dev] = true;
    }
  }
  const long long T = 6LL * n * n * n;
  k_tet_volumes<<<cdiv(T, 256), 256, 0, ex.s>>>(n, X, vol);
  SK_CHECK_LAUNCH();
}

// Half-grid offset (0..2 per axis, packed as ox + 3 oy + 9 oz) of local node a
// of tetrahedron p within its cube (host table, uploaded once).
__constant__ signed char c_tet_node[6][10];
static void upload_tet_nodes() {
  signed char tab[6][10];
  for (int p = 0; p < 6; ++p) {
    int v[4][3];
    ref_tet(p, v);
    for (int a = 0; a < 10; ++a) {
      int q[3];
      for (int c = 0; c < 3; ++c)
        q[c] = a < 4 ? 2 * v[a][c] : v[kEdge[a - 4][0]][c] + v[kEdge[a - 4][1]][c];
      tab[p][a] = (signed char)(q[0] + 3 * q[1] + 9 * q[2]);
    }
  }
  SK_CUDA(cudaMemcpyToSymbol(c_tet_node, tab, sizeof(tab)));
}

// F = M_V f_h with the tet volumes precomputed: one launch per cube colour and
// one thread per (cube, node of the cube's 3x3x3 half-grid block); the thread
// adds the contributions of every tet of the cube that holds its node
// (|K| sum_b M_ab f_b / 420 over the tet's nodes b), tets in order.
__global__ void __launch_bounds__(128) k_load_vol(LoadArgs a, const double* __restrict__ vol) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.mx * a.my * a.mz * 27) return;
  const int nu = t % 27;
  t /= 27;
  const int i = 2 * (t % a.mx) + a.cx;
  const int j = 2 * ((t / a.mx) % a.my) + a.cy;
  const int k = 2 * (t / (a.mx * a.my)) + a.cz;
  const int q[3] = {2 * i + nu % 3, 2 * j + (nu / 3) % 3, 2 * k + nu / 9};
  const int row = p2_interior_index(a.n, q);
  if (row < 0) return;
  const int N = 2 * a.n + 1;
  const size_t base = (size_t)(2 * i) + N * ((size_t)(2 * j) + (size_t)N * (2 * k));
  const size_t cube = (size_t)i + (size_t)a.n * ((size_t)j + (size_t)a.n * k);
  double s[3] = {0, 0, 0};
  for (int p = 0; p < 6; ++p) {
    int la = -1;
    for (int l = 0; l < 10; ++l)
      if (c_tet_node[p][l] == nu) la = l;
    if (la < 0) continue;
    double tp[3] = {0, 0, 0};
    for (int b = 0; b < 10; ++b) {
      const int o = c_tet_node[p][b];
      const size_t gid = base + (size_t)(o % 3) + N * ((size_t)((o / 3) % 3) + (size_t)N * (o / 9));
      const double m = p2_mass420(la, b);
      for (int c = 0; c < 3; ++c) tp[c] += m * a.f[3 * gid + c];
    }
    const double w = vol[6 * cube + p] / 420.0;
    for (int c = 0; c < 3; ++c) s[c] += w * tp[c];
  }
  const size_t nvi = (size_t)(2 * a.n - 1) * (2 * a.n - 1) * (2 * a.n - 1);
  for (int c = 0; c < 3; ++c) a.F[c * nvi + row] += s[c];  // component-major
}

void assemble_load(const Exec& ex, int n, const double* X, const Csr& p2pat, const double* f_all, double* F,
                   const double* vol) {
  if (vol) {
    SK_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * 3 * (size_t)p2pat.rows, ex.s));
    ProfScope ps(ex, STOKES_KERNEL_OTHER, 24.0 * (double)(2 * n + 1) * (2 * n + 1) * (2 * n + 1) + 48.0 * p2pat.rows +
                                              48.0 * n * n * n);
    LoadArgs a{};
    a.n = n;
    a.X = X;
    a.f = f_all;
    a.F = F;
    for (int colour = 0; colour < 8; ++colour) {
      a.cx = colour & 1;
      a.cy = (colour >> 1) & 1;
      a.cz = (colour >> 2) & 1;
      a.mx = (n - a.cx + 1) / 2;
      a.my = (n - a.cy + 1) / 2;
      a.mz = (n - a.cz + 1) / 2;
      const int cubes = a.mx * a.my * a.mz;
      if (cubes == 0) continue;
      k_load_vol<<<cdiv((long long)cubes * 27, 128), 128, 0, ex.s>>>(a, vol);
      if (colour > 0 && ex.prof && ex.prof->on) ex.prof->rec[STOKES_KERNEL_OTHER].launches += 1;
      SK_CHECK_LAUNCH();
    }
    return;
  }
  assemble_load(ex, n, X, p2pat, f_all, F);
}

void assemble_load(const Exec& ex, int n, const double* X, const Csr& p2pat, const double* f_all, double* F) {
  SK_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * 3 * (size_t)p2pat.rows, ex.s));
  ProfScope ps(ex, STOKES_KERNEL_OTHER, 24.0 * (double)(2 * n + 1) * (2 * n + 1) * (2 * n + 1) + 48.0 * p2pat.rows);
  LoadArgs a{};
  a.n = n;
  a.X = X;
  a.f = f_all;
  a.F = F;
  for (int colour = 0; colour < 8; ++colour) {
    a.cx = colour & 1;
    a.cy = (colour >> 1) & 1;
    a.cz = (colour >> 2) & 1;
    a.mx = (n - a.cx + 1) / 2;
    a.my = (n - a.cy + 1) / 2;
    a.mz = (n - a.cz + 1) / 2;
    int cubes = a.mx * a.my * a.mz;
    if (cubes == 0) continue;
    for (int p = 0; p < 6; ++p) {
      a.p = p;
      k_load<<<cdiv((long long)cubes * 10, 128), 128, 0, ex.s>>>(a);
      if ((colour > 0 || p > 0) && ex.prof && ex.prof->on) ex.prof->rec[STOKES_KERNEL_OTHER].launches += 1;
      SK_CHECK_LAUNCH();
    }
  }
}

// out_b += sum_a M_ab lu_a over interior rows a, for all local nodes b (M_V^T lu)
__global__ void __launch_bounds__(128) k_load_t(LoadArgs a) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.mx * a.my * a.mz) return;
  int i = 2 * (t % a.mx) + a.cx;
  int j = 2 * ((t / a.mx) % a.my) + a.cy;
  int k = 2 * (t / (a.mx * a.my)) + a.cz;
  const int N = 2 * a.n + 1;
  for (int p = 0; p < 6; ++p) {
    TetGeom tg;
    tet_geometry(a.n, a.X, i, j, k, p, tg);
    if (!tg.ok) continue;
    int ri[10];
    size_t gid[10];
    double ul[10][3];
    for (int l = 0; l < 10; ++l) {
      int q[3];
      local_node(tg, l, q);
      ri[l] = p2_interior_index(a.n, q);
      gid[l] = (size_t)q[0] + N * ((size_t)q[1] + (size_t)N * q[2]);
      const size_t nvi = (size_t)(2 * a.n - 1) * (2 * a.n - 1) * (2 * a.n - 1);
      for (int c = 0; c < 3; ++c) ul[l][c] = ri[l] >= 0 ? a.f[c * nvi + ri[l]] : 0.0;
    }
    for (int cb = 0; cb < 10; ++cb) {
      double s[3] = {0, 0, 0};
      for (int ra = 0; ra < 10; ++ra) {
        double m = p2_mass420(ra, cb);
        for (int c = 0; c < 3; ++c) s[c] += m * ul[ra][c];
      }
      for (int c = 0; c < 3; ++c) a.F[3 * gid[cb] + c] += tg.vol * s[c] / 420.0;
    }
  }
}

void assemble_load_transpose(const Exec& ex, int n, const double* X, const double* lu, double* out) {
  size_t N = (size_t)(2 * n + 1) * (2 * n + 1) * (2 * n + 1);
  SK_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 3 * N, ex.s));
  LoadArgs a{};
  a.n = n;
  a.X = X;
  a.f = lu;
  a.F = out;
  for (int colour = 0; colour < 8; ++colour) {
    a.cx = colour & 1;
    a.cy = (colour >> 1) & 1;
    a.cz = (colour >> 2) & 1;
    a.mx = (n - a.cx + 1) / 2;
    a.my = (n - a.cy + 1) / 2;
    a.mz = (n - a.cz + 1) / 2;
    int cubes = a.mx * a.my * a.mz;
    if (cubes == 0) continue;
    k_load_t<<<cdiv(cubes, 128), 128, 0, ex.s>>>(a);
    SK_CHECK_LAUNCH();
  }
}

// ---------------------------------------------------------------------------
// multigrid transfers: coarse P2 (P1) functions evaluated at the logical
// (unjittered) positions of fine nodes. On nested Kuhn meshes (nf = 2 nc) this
// is exact interpolation between the nested spaces.
// ---------------------------------------------------------------------------
// Locate point y (coarse-cube units, in [0, nc]^3) in the coarse Kuhn mesh.
__device__ inline void kuhn_locate(int nc, const double y[3], int base[3], int perm[3], double lam[4]) {
  double loc[3];
  for (int c = 0; c < 3; ++c) {
    int b = (int)floor(y[c]);
    b = b < 0 ? 0 : (b > nc - 1 ? nc - 1 : b);
    base[c] = b;
    loc[c] = y[c] - b;
  }
  // axes by decreasing local coordinate (ties by axis index)
  int p0 = 0, p1 = 1, p2 = 2;
  if (loc[p1] > loc[p0]) { int t = p0; p0 = p1; p1 = t; }
  if (loc[p2] > loc[p1]) { int t = p1; p1 = p2; p2 = t; }
  if (loc[p1] > loc[p0]) { int t = p0; p0 = p1; p1 = t; }
  perm[0] = p0; perm[1] = p1; perm[2] = p2;
  lam[0] = 1.0 - loc[p0];
  lam[1] = loc[p0] - loc[p1];
  lam[2] = loc[p1] - loc[p2];
  lam[3] = loc[p2];
}

__device__ inline void kuhn_vertices_of(const int base[3], const int perm[3], int v[4][3]) {
  for (int c = 0; c < 3; ++c) {
    v[0][c] = base[c];
    v[1][c] = base[c] + (c == perm[0]);
    v[2][c] = v[1][c] + (c == perm[1]);
    v[3][c] = base[c] + 1;
  }
}

// P2 weights of the coarse interior nodes at fine half-grid node qf; returns count.
__device__ inline int p2_interp(int nf, int nc, const int qf[3], int node[10], double w[10]) {
  double y[3];
  for (int c = 0; c < 3; ++c) y[c] = (double)qf[c] * nc / (2.0 * nf);
  int base[3], perm[3], v[4][3];
  double lam[4];
  kuhn_locate(nc, y, base, perm, lam);
  kuhn_vertices_of(base, perm, v);
  int cnt = 0;
  for (int a = 0; a < 10; ++a) {
    int q[3];
    double wt;
    if (a < 4) {
      for (int c = 0; c < 3; ++c) q[c] = 2 * v[a][c];
      wt = lam[a] * (2.0 * lam[a] - 1.0);
    } else {
      int l = c_edge[a - 4][0], m = c_edge[a - 4][1];
      for (int c = 0; c < 3; ++c) q[c] = v[l][c] + v[m][c];
      wt = 4.0 * lam[l] * lam[m];
    }
    int id = p2_interior_index(nc, q);
    if (id < 0 || fabs(wt) < 1e-13) continue;
    node[cnt] = id;
    w[cnt] = wt;
    ++cnt;
  }
  return cnt;
}

__device__ inline int p1_interp(int nf, int nc, const int vf[3], int node[4], double w[4]) {
  double y[3];
  for (int c = 0; c < 3; ++c) y[c] = (double)vf[c] * nc / (double)nf;
  int base[3], perm[3], v[4][3];
  double lam[4];
  kuhn_locate(nc, y, base, perm, lam);
  kuhn_vertices_of(base, perm, v);
  int cnt = 0;
  for (int l = 0; l < 4; ++l) {
    if (fabs(lam[l]) < 1e-13) continue;
    node[cnt] = v[l][0] + (nc + 1) * (v[l][1] + (nc + 1) * v[l][2]);
    w[cnt] = lam[l];
    ++cnt;
  }
  return cnt;
}

__global__ void k_prolong_rows(int pass, int p2, int nf, int nc, int* __restrict__ cnt_or_rp,
                               int* __restrict__ col, double* __restrict__ val) {
  int e = p2 ? 2 * nf - 1 : nf + 1;
  int lo = p2 ? 1 : 0;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= e * e * e) return;
  int q[3] = {lo + r % e, lo + (r / e) % e, lo + r / (e * e)};
  int node[10];
  double w[10];
  int c = p2 ? p2_interp(nf, nc, q, node, w) : p1_interp(nf, nc, q, node, w);
  if (!pass) {
    cnt_or_rp[r] = c;
    return;
  }
  int o = cnt_or_rp[r];
  for (int t = 0; t < c; ++t) col[o + t] = node[t], val[o + t] = w[t];
}

// rows of R = P^T: for coarse node Q, scan the fine nodes inside its support
__global__ void k_restrict_rows(int pass, int p2, int nf, int nc, int* __restrict__ cnt_or_rp,
                                int* __restrict__ col, double* __restrict__ val) {
  int ec = p2 ? 2 * nc - 1 : nc + 1;
  int lo = p2 ? 1 : 0;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ec * ec * ec) return;
  int Q[3] = {lo + r % ec, lo + (r / ec) % ec, lo + r / (ec * ec)};
  // support of the coarse basis function: |x - x_Q| <= 1/nc (logical units)
  int fl[3], fh[3];
  int scale_f = p2 ? 2 * nf : nf, scale_c = p2 ? 2 * nc : nc;
  int reach = p2 ? 2 : 1;  // one coarse cell in coarse index units
  int ef = p2 ? 2 * nf - 1 : nf + 1;
  for (int c = 0; c < 3; ++c) {
    long long a = (long long)(Q[c] - reach) * scale_f, b = (long long)(Q[c] + reach) * scale_f;
    long long l = a >= 0 ? (a + scale_c - 1) / scale_c : -((-a) / scale_c);
    long long h = b >= 0 ? b / scale_c : -((-b + scale_c - 1) / scale_c);
    fl[c] = (int)max((long long)lo, l);
    fh[c] = (int)min((long long)(lo + ef - 1), h);
  }
  int o = pass ? cnt_or_rp[r] : 0, count = 0;
  for (int z = fl[2]; z <= fh[2]; ++z)
    for (int y = fl[1]; y <= fh[1]; ++y)
      for (int x = fl[0]; x <= fh[0]; ++x) {
        int q[3] = {x, y, z};
        int node[10];
        double w[10];
        int c = p2 ? p2_interp(nf, nc, q, node, w) : p1_interp(nf, nc, q, node, w);
        for (int t = 0; t < c; ++t)
          if (node[t] == r) {
            if (pass) {
              col[o] = (x - lo) + ef * ((y - lo) + ef * (z - lo));
              val[o] = w[t];
              ++o;
            } else {
              ++count;
            }
          }
      }
  if (!pass) cnt_or_rp[r] = count;
}

static void build_transfer(const Exec& ex, Arena& ar, int p2, int nf, int nc, Csr& P, Csr& R) {
  int ef = p2 ? 2 * nf - 1 : nf + 1, ec = p2 ? 2 * nc - 1 : nc + 1;
  long long rf = (long long)ef * ef * ef, rc = (long long)ec * ec * ec;
  for (int which = 0; which < 2; ++which) {
    Csr& m = which == 0 ? P : R;
    long long rows = which == 0 ? rf : rc;
    m.rows = (int)rows;
    m.cols = (int)(which == 0 ? rc : rf);
    m.rowptr = ar.alloc<int>(rows + 1);
    int* cnt = ar.alloc<int>(rows);
    int nb = cdiv(rows, 128);
    if (which == 0)
      k_prolong_rows<<<nb, 128, 0, ex.s>>>(0, p2, nf, nc, cnt, nullptr, nullptr);
    else
      k_restrict_rows<<<nb, 128, 0, ex.s>>>(0, p2, nf, nc, cnt, nullptr, nullptr);
    SK_CHECK_LAUNCH();
    long long total;
    scan_counts(ex, ar, cnt, m.rows, m.rowptr, &total);
    m.nnz = total;
    m.col = ar.alloc<int>(total);
    m.v64 = ar.alloc<double>(total);
    if (which == 0)
      k_prolong_rows<<<nb, 128, 0, ex.s>>>(1, p2, nf, nc, m.rowptr, m.col, m.v64);
    else
      k_restrict_rows<<<nb, 128, 0, ex.s>>>(1, p2, nf, nc, m.rowptr, m.col, m.v64);
    SK_CHECK_LAUNCH();
  }
}

void build_transfer_p2(const Exec& ex, Arena& ar, int nf, int nc, Csr& P, Csr& R) {
  build_transfer(ex, ar, 1, nf, nc, P, R);
}
void build_transfer_p1(const Exec& ex, Arena& ar, int nf, int nc, Csr& P, Csr& R) {
  build_transfer(ex, ar, 0, nf, nc, P, R);
}

// ---------------------------------------------------------------------------
__global__ void k_diag_inv(int rows, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ v, double* __restrict__ dinv) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  int pos = find_col(col, rp[r], rp[r + 1], r);
  dinv[r] = pos >= 0 ? 1.0 / v[pos] : 0.0;
}

__global__ void k_diag_inv3(int rows, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ v, long long nnz, double* __restrict__ dinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  int pos = find_col(col, rp[i], rp[i + 1], i);
  for (int r = 0; r < 3; ++r) {
    const double a = pos >= 0 ? v[(size_t)(4 * r) * nnz + pos] : 0.0;  // plane 3r + r
    dinv[(size_t)r * rows + i] = a != 0.0 ? 1.0 / a : 0.0;
  }
}

void diag_inverse(const Exec& ex, const Csr& m, double* dinv) {
  if (m.br == 3) {
    k_diag_inv3<<<cdiv(m.rows, 256), 256, 0, ex.s>>>(m.rows, m.rowptr, m.col, m.v64, m.nnz, dinv);
  } else {
    k_diag_inv<<<cdiv(m.rows, 256), 256, 0, ex.s>>>(m.rows, m.rowptr, m.col, m.v64, dinv);
  }
  SK_CHECK_LAUNCH();
}

// A~_1 = A + g mu D with mu D = A - A~_3 (x) I on interior velocities (E_V =
// L_V + D on H^1_0): (1 + g) A - g A~_3 on the diagonal planes 0, 4, 8
__global__ void k_combine_grad_div(long long nnz, const double* __restrict__ abs, const double* __restrict__ a3,
                                   double g, double* __restrict__ out) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz;
       k += (long long)gridDim.x * blockDim.x)
    for (int j = 0; j < 9; ++j) {
      const size_t i = (size_t)j * nnz + k;
      out[i] = (1.0 + g) * abs[i] - ((j % 4) == 0 ? g * a3[k] : 0.0);
    }
}

void combine_grad_div(const Exec& ex, long long nnz, const double* abs, const double* a3, double g, double* out) {
  if (!nnz) return;
  k_combine_grad_div<<<(int)std::min<long long>(cdiv(nnz, 256), 4096), 256, 0, ex.s>>>(nnz, abs, a3, g, out);
  SK_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// stencil-structured storage (see StencilOp in internal.h)
// ---------------------------------------------------------------------------
StArgs stencil_args(const StencilOp& so, int block, int rows_per_thread, bool split) {
  StArgs a;
  std::memset(&a, 0, sizeof(a));
  a.p2 = so.p2;
  a.split = split && so.p2 ? 1 : 0;
  a.n = so.n;
  a.ncls = so.ncls;
  a.lo = so.p2 ? 1 : 0;
  a.hi = so.p2 ? 2 * so.n - 1 : 2 * so.n;
  a.m = so.p2 ? 2 * so.n - 1 : so.n + 1;
  a.R = rows_per_thread;
  int b = 0;
  for (int c = 0; c < so.ncls; ++c) {
    a.rows[c] = so.rows[c];
    a.S[c] = so.S[c];
    a.Sreal[c] = so.Sreal[c];
    a.dbeg[c] = so.dbeg[c];
    a.voff[c] = so.voff[c];
    a.pext[c] = so.pext[c];
    a.prows[c] = so.prows[c];
    for (int k = 0; k < 3; ++k) a.ext[c][k] = so.ext[c][k], a.q0[c][k] = so.q0[c][k];
    a.bbeg[c] = b;
    b += cdiv(so.prows[c] / rows_per_thread, block);
  }
  a.bbeg[so.ncls] = b;
  for (int e = 0; e < so.nd; ++e) {
    for (int k = 0; k < 3; ++k) a.d[e][k] = so.d[e][k];
    a.lin[e] = a.split ? so.lin_split[e] : so.lin[e];
  }
  return a;
}

// one thread per padded row: values of entry e at
// voff[c] + ((e / kStencilVec) * prows[c] + pr) * kStencilVec + e % kStencilVec
__global__ void k_stencil_fill(const StArgs a, const int* __restrict__ rp, const int* __restrict__ col,
                               const double* __restrict__ val, double* __restrict__ out) {
  int c, pr;
  if (!st_locate(a, c, pr)) return;
  int i, qx, qy, qz;
  st_coords(a, c, pr, i, qx, qy, qz);
  const bool real = i < a.ext[c][0];
  const int row = real ? st_index(a, qx, qy, qz) : 0;
  const int lo = real ? rp[row] : 0, hi = real ? rp[row + 1] : 0;
  for (int e = 0; e < a.S[c]; ++e) {
    const int de = a.dbeg[c] + e;
    double w = 0.0;
    if (real && e < a.Sreal[c] && st_inside(a, qx + a.d[de][0], qy + a.d[de][1], qz + a.d[de][2])) {
      int pos = find_col(col, lo, hi, row + a.lin[de]);
      if (pos >= 0) w = val[pos];
    }
    out[a.voff[c] + ((size_t)(e / kStencilVec) * a.prows[c] + pr) * kStencilVec + e % kStencilVec] = w;
  }
}

StencilOp* stencil_from_csr(const Exec& ex, Arena& ar, const StencilTables* st, int p2, int n, const Csr& m) {
  SK_REQUIRE(m.br == 1 && m.bc == 1 && m.v64, STOKES_ERR_ARG, "stencil storage needs a scalar FP64 CSR matrix");
  auto* so = new StencilOp();
  so->p2 = p2;
  so->n = n;
  so->ncls = p2 ? 8 : 1;
  const int kind = p2 ? PAT_P2P2 : PAT_P1P1;
  const int mm = p2 ? 2 * n - 1 : n + 1;
  long long off = 0;
  int nd = 0;
  for (int c = 0; c < so->ncls; ++c) {
    for (int k = 0; k < 3; ++k) {
      int par = p2 ? ((c >> k) & 1) : 0;
      so->q0[c][k] = p2 ? (par ? 1 : 2) : 0;
      so->ext[c][k] = p2 ? (par ? n : n - 1) : n + 1;
    }
    so->rows[c] = so->ext[c][0] * so->ext[c][1] * so->ext[c][2];
    so->pext[c] = (so->ext[c][0] + kStencilRows - 1) / kStencilRows * kStencilRows;
    so->prows[c] = so->pext[c] * so->ext[c][1] * so->ext[c][2];
    so->dbeg[c] = nd;
    const int s0 = st->beg[kind][c], s1 = st->beg[kind][c + 1];
    const int padded = (s1 - s0 + kStencilVec - 1) / kStencilVec * kStencilVec;
    for (int k = 0; k < padded; ++k) {
      SK_REQUIRE(nd < kMaxStencil, STOKES_ERR_ARG, "stencil table overflow");
      int dx = 0, dy = 0, dz = 0;  // padding entries: offset 0, weight 0
      if (s0 + k < s1) dx = st->h_off[3 * (s0 + k)], dy = st->h_off[3 * (s0 + k) + 1], dz = st->h_off[3 * (s0 + k) + 2];
      so->d[nd][0] = (signed char)dx;
      so->d[nd][1] = (signed char)dy;
      so->d[nd][2] = (signed char)dz;
      so->lin[nd] = p2 ? dx + mm * (dy + mm * dz) : dx / 2 + mm * (dy / 2 + mm * (dz / 2));
      if (p2) {
        // parity-split numbering: a row of this class has x-index t of parity
        // px; its neighbour t + dx has parity (px + dx) mod 2 and sits
        // floor((px + dx) / 2) places further along its half of the line
        const int px = (so->q0[c][0] - 1) & 1;
        const int pn = ((px + dx) % 2 + 2) % 2;
        const int fx = (px + dx + 4) / 2 - 2;
        so->lin_split[nd] = (pn - px) * n + fx + mm * (dy + mm * dz);
      }
      ++nd;
    }
    so->S[c] = nd - so->dbeg[c];
    so->Sreal[c] = s1 - s0;
    so->total_real += (long long)so->Sreal[c] * so->prows[c];
    so->voff[c] = off;
    off += (long long)so->S[c] * so->prows[c];
  }
  so->nd = nd;
  so->total = off;
  long long rows_all = 0;
  for (int c = 0; c < so->ncls; ++c) rows_all += so->rows[c];
  SK_REQUIRE(off < (1LL << 32) && 3 * rows_all < (1LL << 32), STOKES_ERR_ARG,
             "stencil storage needs 32-bit indices (mesh too large)");
  so->v64 = ar.alloc<double>(off);
  StArgs a = stencil_args(*so, 128, 1);
  k_stencil_fill<<<a.bbeg[so->ncls], 128, 0, ex.s>>>(a, m.rowptr, m.col, m.v64, so->v64);
  SK_CHECK_LAUNCH();
  return so;
}

// ---------------------------------------------------------------------------
// symmetric stencil storage of a BSR3 interior-P2 matrix (see Sym3Op)
// ---------------------------------------------------------------------------
struct Sym3Fill {
  int n, m;
  int ext[8][3], q0[8][3], pext[8], prows[8], ubeg[9], bbeg[9];
  long long voff[8];
  signed char ud[kMaxSym][3];
  int ulin[kMaxSym];
};

// one thread per padded row of one class; block e, entry k of row pr at
// voff[c] + (9 e + k) prows[c] + pr
__global__ void k_sym3_fill(const Sym3Fill a, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ val, long long nnz, double* __restrict__ out) {
  int c = 0;
  while (c < 7 && (int)blockIdx.x >= a.bbeg[c + 1]) ++c;
  const int pr = ((int)blockIdx.x - a.bbeg[c]) * (int)blockDim.x + (int)threadIdx.x;
  if (pr >= a.prows[c]) return;
  const int px = a.pext[c], ey = a.ext[c][1];
  const int i = pr % px;
  const int qx = a.q0[c][0] + 2 * i, qy = a.q0[c][1] + 2 * ((pr / px) % ey), qz = a.q0[c][2] + 2 * (pr / (px * ey));
  const bool real = i < a.ext[c][0];
  const int row = real ? (qx - 1) + a.m * ((qy - 1) + a.m * (qz - 1)) : 0;
  const int lo = real ? rp[row] : 0, hi = real ? rp[row + 1] : 0;
  const int hiq = 2 * a.n - 1;
  for (int e = a.ubeg[c]; e < a.ubeg[c + 1]; ++e) {
    const int jx = qx + a.ud[e][0], jy = qy + a.ud[e][1], jz = qz + a.ud[e][2];
    int pos = -1;
    if (real && jx >= 1 && jx <= hiq && jy >= 1 && jy <= hiq && jz >= 1 && jz <= hiq)
      pos = find_col(col, lo, hi, row + a.ulin[e]);
    const size_t base = (size_t)a.voff[c] + (size_t)9 * (e - a.ubeg[c]) * a.prows[c] + pr;
    for (int k = 0; k < 9; ++k) out[base + (size_t)k * a.prows[c]] = pos >= 0 ? val[(size_t)k * nnz + pos] : 0.0;
  }
}

Sym3Op* sym3_from_csr(const Exec& ex, Arena& ar, const StencilTables* st, int n, const Csr& m) {
  SK_REQUIRE(m.br == 3 && m.bc == 3 && m.v64, STOKES_ERR_ARG, "symmetric stencil storage needs an FP64 BSR3 matrix");
  SK_REQUIRE(n >= 2, STOKES_ERR_ARG, "symmetric stencil storage needs n >= 2");
  auto* so = new Sym3Op();
  so->n = n;
  const int mm = 2 * n - 1;
  for (int c = 0; c < 8; ++c) {
    for (int k = 0; k < 3; ++k) {
      const int par = (c >> k) & 1;
      so->q0[c][k] = par ? 1 : 2;
      so->ext[c][k] = par ? n : n - 1;
    }
    so->rows[c] = so->ext[c][0] * so->ext[c][1] * so->ext[c][2];
    so->pext[c] = so->ext[c][0];
    so->prows[c] = so->rows[c];
  }
  // lexicographic sign in (z, y, x): the sign of the linear offset for m >= 3
  auto lex = [](int dx, int dy, int dz) { return dz != 0 ? dz : (dy != 0 ? dy : dx); };
  auto lin = [&](int dx, int dy, int dz) { return dx + mm * (dy + mm * dz); };
  std::vector<std::vector<std::array<int, 3>>> up(8), low(8);
  for (int c = 0; c < 8; ++c) {
    up[c].push_back({0, 0, 0});
    for (int e = st->beg[PAT_P2P2][c]; e < st->beg[PAT_P2P2][c + 1]; ++e) {
      std::array<int, 3> o{st->h_off[3 * e], st->h_off[3 * e + 1], st->h_off[3 * e + 2]};
      const int sg = lex(o[0], o[1], o[2]);
      if (sg > 0) up[c].push_back(o);
      else if (sg < 0) low[c].push_back(o);
    }
  }
  int nu = 0, nl = 0;
  long long off = 0;
  for (int c = 0; c < 8; ++c) {
    so->ubeg[c] = nu;
    for (auto& o : up[c]) {
      SK_REQUIRE(nu < kMaxSym, STOKES_ERR_ARG, "symmetric stencil table overflow");
      for (int k = 0; k < 3; ++k) so->ud[nu][k] = (signed char)o[k];
      so->ulin[nu] = lin(o[0], o[1], o[2]);
      ++nu;
    }
    so->voff[c] = off;
    off += 9LL * (long long)up[c].size() * so->prows[c];
  }
  so->ubeg[8] = nu;
  for (int c = 0; c < 8; ++c) {
    so->lbeg[c] = nl;
    for (auto& o : low[c]) {
      SK_REQUIRE(nl < kMaxSym, STOKES_ERR_ARG, "symmetric stencil table overflow");
      const int cs = c ^ ((o[0] & 1) | ((o[1] & 1) << 1) | ((o[2] & 1) << 2));
      int es = -1;
      for (size_t e = 0; e < up[cs].size(); ++e)
        if (up[cs][e][0] == -o[0] && up[cs][e][1] == -o[1] && up[cs][e][2] == -o[2]) es = (int)e;
      SK_REQUIRE(es >= 0, STOKES_ERR_ARG, "stencil pattern is not symmetric");
      for (int k = 0; k < 3; ++k) {
        so->ld[nl][k] = (signed char)o[k];
        const int t = so->q0[c][k] + o[k] - so->q0[cs][k];
        SK_REQUIRE((t & 1) == 0, STOKES_ERR_ARG, "stencil class parity mismatch");
        so->ldel[nl][k] = (signed char)(t / 2);
      }
      so->llin[nl] = lin(o[0], o[1], o[2]);
      so->lcls[nl] = cs;
      so->lbase[nl] = so->voff[cs] + 9LL * es * so->prows[cs];
      ++nl;
    }
  }
  so->lbeg[8] = nl;
  so->total = off;
  SK_REQUIRE(off < (1LL << 40), STOKES_ERR_ARG, "symmetric stencil storage too large");
  so->v64 = ar.alloc<double>(off);
  Sym3Fill a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.m = mm;
  int b = 0;
  for (int c = 0; c < 8; ++c) {
    for (int k = 0; k < 3; ++k) a.ext[c][k] = so->ext[c][k], a.q0[c][k] = so->q0[c][k];
    a.pext[c] = so->pext[c];
    a.prows[c] = so->prows[c];
    a.voff[c] = so->voff[c];
    a.ubeg[c] = so->ubeg[c];
    a.bbeg[c] = b;
    b += cdiv(so->prows[c], 128);
  }
  a.ubeg[8] = so->ubeg[8];
  a.bbeg[8] = b;
  for (int e = 0; e < nu; ++e) {
    for (int k = 0; k < 3; ++k) a.ud[e][k] = so->ud[e][k];
    a.ulin[e] = so->ulin[e];
  }
  if (b > 0) {
    k_sym3_fill<<<b, 128, 0, ex.s>>>(a, m.rowptr, m.col, m.v64, m.nnz, so->v64);
    SK_CHECK_LAUNCH();
  }
  return so;
}

__global__ void k_to_f32(const double* __restrict__ s, float* __restrict__ d, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (float)s[i];
}

void to_f32(const Exec& ex, const double* src, float* dst, size_t n) {
  if (!n) return;
  k_to_f32<<<cdiv(n, 256), 256, 0, ex.s>>>(src, dst, n);
  SK_CHECK_LAUNCH();
}

__global__ void k_to_f32_lo(const double* __restrict__ s, const float* __restrict__ hi, float* __restrict__ lo,
                            size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    lo[i] = (float)(s[i] - (double)hi[i]);
}

void to_f32_lo(const Exec& ex, const double* src, const float* hi, float* lo, size_t n) {
  if (!n) return;
  k_to_f32_lo<<<(unsigned)std::min<size_t>(cdiv(n, 256), 1 << 20), 256, 0, ex.s>>>(src, hi, lo, n);
  SK_CHECK_LAUNCH();
}

// Coarse-level geometry: coarse vertex i sits at logical position i/nc; its
// coordinates are the P1 interpolation of the fine (jittered) vertex
// positions at that logical point on the fine Kuhn mesh. For nf = 2 nc this is
// exactly the fine vertex 2i; for other ratios it is a smooth average of the
// fine jitter, so coarse tetrahedra are no more distorted than fine ones.
void subsample_vertices(int nf, int nc, const double* Xf, double* Xc) {
  const int nvf = nf + 1, nvc = nc + 1;
  for (int k = 0; k <= nc; ++k)
    for (int j = 0; j <= nc; ++j)
      for (int i = 0; i <= nc; ++i) {
        const int ic[3] = {i, j, k};
        int base[3];
        double t[3];
        for (int c = 0; c < 3; ++c) {
          // y = ic * nf / nc in fine-cube units, exactly when the ratio is integral
          long long num = (long long)ic[c] * nf;
          int b = (int)(num / nc);
          if (b > nf - 1) b = nf - 1;
          base[c] = b;
          t[c] = (double)(num - (long long)b * nc) / nc;
        }
        int p0 = 0, p1 = 1, p2 = 2;  // axes by decreasing local coordinate
        if (t[p1] > t[p0]) std::swap(p0, p1);
        if (t[p2] > t[p1]) std::swap(p1, p2);
        if (t[p1] > t[p0]) std::swap(p0, p1);
        const double lam[4] = {1.0 - t[p0], t[p0] - t[p1], t[p1] - t[p2], t[p2]};
        int v[4][3];
        for (int c = 0; c < 3; ++c) {
          v[0][c] = base[c];
          v[1][c] = base[c] + (c == p0);
          v[2][c] = v[1][c] + (c == p1);
          v[3][c] = base[c] + 1;
        }
        const size_t cc = (size_t)i + nvc * ((size_t)j + (size_t)nvc * k);
        for (int c = 0; c < 3; ++c) {
          double x = 0.0;
          for (int l = 0; l < 4; ++l) {
            if (lam[l] == 0.0) continue;
            size_t fv = (size_t)v[l][0] + nvf * ((size_t)v[l][1] + (size_t)nvf * v[l][2]);
            x += lam[l] * Xf[3 * fv + c];
          }
          Xc[3 * cc + c] = x;
        }
      }
}

}  // namespace sk
