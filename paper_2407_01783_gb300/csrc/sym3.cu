// Products with the strain-form velocity operator A in symmetric stencil
// storage (Sym3Op): each row reads its diagonal and "upper" 3x3 blocks from its
// own storage and the transposes of its "lower" blocks from the neighbours'
// storage, so the stored values are half of the BSR3 values and carry no
// column indices.
//
// Launch order: blocks walk the half-grid z-planes in order and, within a
// plane, the four classes that have rows there. A lower block of row i
// (neighbour j at most one cube layer below i) was read directly by row j a
// few planes earlier, i.e. within the last few tens of MB of traffic, so the
// second read is served from L2 and each value crosses HBM about once.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace sk {

struct Sym3Args {
  int m, hiq;                  // points per axis (2n-1); highest interior half-grid coordinate
  int bo, be;                  // blocks of an odd / even half-grid z-plane (all its classes)
  int nb[8];                   // blocks per (class, plane)
  int ext[8][3], q0[8][3], pext[8], prows[8], ubeg[9], lbeg[9];
  long long voff[8];
  signed char ud[kMaxSym][3];
  int ulin[kMaxSym];
  signed char ld[kMaxSym][3];
  int llin[kMaxSym];
  int lcls[kMaxSym];
  long long lbase[kMaxSym];
  signed char ldel[kMaxSym][3];
};

constexpr int kSymBlock = 128;

// G threads share a row (G in {1, 2, 4, 8}), so a block covers 128 / G rows
static Sym3Args sym3_args(const Sym3Op& so, int G) {
  Sym3Args a;
  std::memset(&a, 0, sizeof(a));
  a.m = 2 * so.n - 1;
  a.hiq = 2 * so.n - 1;
  const int rows_per_block = kSymBlock / G;
  for (int c = 0; c < 8; ++c) {
    for (int k = 0; k < 3; ++k) a.ext[c][k] = so.ext[c][k], a.q0[c][k] = so.q0[c][k];
    a.pext[c] = so.pext[c];
    a.prows[c] = so.prows[c];
    a.voff[c] = so.voff[c];
    a.nb[c] = cdiv((long long)so.pext[c] * so.ext[c][1], rows_per_block);
  }
  for (int c = 0; c < 9; ++c) a.ubeg[c] = so.ubeg[c], a.lbeg[c] = so.lbeg[c];
  // classes with an odd z coordinate (bit 2 set) have rows on odd planes
  a.bo = a.nb[4] + a.nb[5] + a.nb[6] + a.nb[7];
  a.be = a.nb[0] + a.nb[1] + a.nb[2] + a.nb[3];
  for (int e = 0; e < so.ubeg[8]; ++e) {
    for (int k = 0; k < 3; ++k) a.ud[e][k] = so.ud[e][k];
    a.ulin[e] = so.ulin[e];
  }
  for (int e = 0; e < so.lbeg[8]; ++e) {
    for (int k = 0; k < 3; ++k) a.ld[e][k] = so.ld[e][k], a.ldel[e][k] = so.ldel[e][k];
    a.llin[e] = so.llin[e];
    a.lcls[e] = so.lcls[e];
    a.lbase[e] = so.lbase[e];
  }
  return a;
}

// n odd planes (qz = 1, 3, ..., 2n-1) and n-1 even planes (qz = 2, ..., 2n-2),
// interleaved: odd plane k, even plane k, odd plane k+1, ...
static int sym3_blocks(const Sym3Op& so, const Sym3Args& a) { return so.n * a.bo + (so.n - 1) * a.be; }
// most blocks any thread-per-row width launches (8 threads per row)
int sym3_grid(const Sym3Op& so) { return sym3_blocks(so, sym3_args(so, 8)); }

struct SymRow {
  int c, ix, iy, iz, pr, row, qx, qy, qz;
  bool valid;
};

template <int G>
__device__ __forceinline__ SymRow sym3_locate(const Sym3Args& a, int vb) {
  SymRow r;
  const int pair = vb / (a.bo + a.be);
  int rem = vb - pair * (a.bo + a.be);
  const bool odd = rem < a.bo;
  if (!odd) rem -= a.bo;
  int c = odd ? 4 : 0;
#pragma unroll 1
  for (int k = 0; k < 3 && rem >= a.nb[c]; ++k) rem -= a.nb[c++];
  r.c = c;
  r.iz = pair;  // odd planes: qz = 1 + 2 pair; even planes: qz = 2 + 2 pair
  const int plane = a.pext[c] * a.ext[c][1];
  const int t = rem * (kSymBlock / G) + (int)threadIdx.x / G;
  r.valid = t < plane;
  const int tt = r.valid ? t : 0;
  r.ix = tt % a.pext[c];
  r.iy = tt / a.pext[c];
  r.pr = r.iz * plane + tt;
  r.qx = a.q0[c][0] + 2 * r.ix;
  r.qy = a.q0[c][1] + 2 * r.iy;
  r.qz = a.q0[c][2] + 2 * r.iz;
  r.row = (r.qx - 1) + a.m * ((r.qy - 1) + a.m * (r.qz - 1));
  return r;
}

__device__ __forceinline__ bool sym3_inside(const Sym3Args& a, int x, int y, int z) {
  return x >= 1 && x <= a.hiq && y >= 1 && y <= a.hiq && z >= 1 && z <= a.hiq;
}

// Batched loads (as in the CSR kernels): a lane first issues the value loads
// of U entries (entries lane, lane + G, ..., lane + (U-1) G of its row), then
// their x gathers, then the FMAs, so that U block loads per lane are in flight
// per HBM round trip. Entries past the end re-read a valid entry and weigh 0.
template <int G>
struct SymBatch {
  static constexpr int U = 8 / G;
};

// this lane's share of acc[3k + r] = sum over the row's blocks of
// A(i, j)_{r q} x_k,j[q] for K right-hand sides (x: 3K component-major
// components), U entries' loads in flight per lane; each block is read once
// for all K
template <int G, int U, int K, class T>
__device__ __forceinline__ void sym3_row(const Sym3Args& a, const SymRow& R, int lane, const T* __restrict__ v,
                                         const T* __restrict__ x, size_t xs, T* acc) {
  const int c = R.c;
  const int last = (int)xs - 1;
  const size_t rc = (size_t)a.prows[c];
  const T* vr = v + a.voff[c] + R.pr;
  const int u0 = a.ubeg[c], nu = a.ubeg[c + 1] - u0;
  for (int e0 = lane; e0 < nu; e0 += U * G) {
    T w[U][9];
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * G;
      const bool ok = e < nu;
      const int es = ok ? e : nu - 1;
      cc[u] = min(max(R.row + a.ulin[u0 + es], 0), last);
      const T* vb = vr + (size_t)9 * es * rc;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const T t = vb[k * rc];
        w[u][k] = ok ? t : T(0);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T* xk = x + (size_t)3 * k * xs;
      T xv[U][3];
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u][0] = xk[cc[u]], xv[u][1] = xk[xs + cc[u]], xv[u][2] = xk[2 * xs + cc[u]];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          acc[3 * k + r] += w[u][3 * r] * xv[u][0] + w[u][3 * r + 1] * xv[u][1] + w[u][3 * r + 2] * xv[u][2];
    }
  }
  const int l0 = a.lbeg[c], nl = a.lbeg[c + 1] - l0;
  for (int e0 = lane; e0 < nl; e0 += U * G) {
    T w[U][9];
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * G;
      const int L = l0 + (e < nl ? e : nl - 1);
      const bool in = e < nl && sym3_inside(a, R.qx + a.ld[L][0], R.qy + a.ld[L][1], R.qz + a.ld[L][2]);
      const int cs = a.lcls[L];
      const int jx = R.ix + a.ldel[L][0], jy = R.iy + a.ldel[L][1], jz = R.iz + a.ldel[L][2];
      const int rj = in ? jx + a.pext[cs] * (jy + a.ext[cs][1] * jz) : 0;
      const size_t rcs = (size_t)a.prows[cs];
      const T* vb = v + a.lbase[L] + rj;
      cc[u] = min(max(R.row + a.llin[L], 0), last);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const T t = vb[k * rcs];
        w[u][k] = in ? t : T(0);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T* xk = x + (size_t)3 * k * xs;
      T xv[U][3];
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u][0] = xk[cc[u]], xv[u][1] = xk[xs + cc[u]], xv[u][2] = xk[2 * xs + cc[u]];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          acc[3 * k + r] += w[u][r] * xv[u][0] + w[u][3 + r] * xv[u][1] + w[u][6 + r] * xv[u][2];
    }
  }
}

// y = A x (b == nullptr) or y = b - A x; with DOT, *dot = x . (A x) over all rows
// Blocks walk the virtual blocks (plane order) with a grid stride; the dot
// variant runs one resident wave so that its grid sum takes one counter
// increment per resident block.
// K right-hand sides: x, b, y hold 3K component-major components (the dot
// variant is K = 1 only)
template <int G, int U, class T, bool DOT, int K = 1>
__global__ void __launch_bounds__(kSymBlock) k_sym3(const Sym3Args a, int nvb, const T* __restrict__ v,
                                                   const T* __restrict__ x, size_t xs, const T* __restrict__ b,
                                                   T* __restrict__ y, double* partial, unsigned* counter,
                                                   double* dot) {
  static_assert(!DOT || K == 1, "fused dot: one right-hand side");
  const int lane = (int)threadIdx.x % G;
  double part = 0.0;
  for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const SymRow R = sym3_locate<G>(a, vb);
    T acc[3 * K];
#pragma unroll
    for (int r = 0; r < 3 * K; ++r) acc[r] = T(0);
    if (R.valid) sym3_row<G, U, K, T>(a, R, lane, v, x, xs, acc);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < 3 * K; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (R.valid && lane == 0) {
#pragma unroll
      for (int r = 0; r < 3 * K; ++r) {
        const size_t i = r * xs + R.row;
        y[i] = b ? b[i] - acc[r] : acc[r];
        if (DOT) part += (double)(acc[r] * x[i]);
      }
    }
  }
  if (DOT) grid_sum(part, partial, counter, dot);
}

// y = b - A x in double-float arithmetic: A = vh + vl, x = xh + xl (FP32
// pairs); K right-hand sides (x, b, y: 3K component-major components), each
// stored block read once for all K
template <int G, int K = 1>
__global__ void __launch_bounds__(kSymBlock) k_sym3_df(const Sym3Args a, const float* __restrict__ vh,
                                                      const float* __restrict__ vl, const float* __restrict__ xh,
                                                      const float* __restrict__ xl, size_t xs,
                                                      const double* __restrict__ b, double* __restrict__ y) {
  const SymRow R = sym3_locate<G>(a, (int)blockIdx.x);
  const int lane = (int)threadIdx.x % G;
  const int c = R.c;
  const int last = (int)xs - 1;
  DF acc[3 * K];
#pragma unroll
  for (int r = 0; r < 3 * K; ++r) acc[r] = DF{0.f, 0.f};
  constexpr int U = K > 1 ? 1 : (SymBatch<G>::U > 4 ? 4 : SymBatch<G>::U);
  if (R.valid) {
    const size_t rc = (size_t)a.prows[c];
    const int u0 = a.ubeg[c], nu = a.ubeg[c + 1] - u0;
    for (int e0 = lane; e0 < nu; e0 += U * G) {
      float wh[U][9], wl[U][9];
      int cc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * G;
        const bool ok = e < nu;
        const int es = ok ? e : nu - 1;
        cc[u] = min(max(R.row + a.ulin[u0 + es], 0), last);
        const size_t base = a.voff[c] + (size_t)9 * es * rc + R.pr;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const float h = vh[base + k * rc], l = vl[base + k * rc];
          wh[u][k] = ok ? h : 0.f;
          wl[u][k] = ok ? l : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float x_h[3], x_l[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) x_h[q] = xh[(3 * k + q) * xs + cc[u]], x_l[q] = xl[(3 * k + q) * xs + cc[u]];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q)
              df_madd(acc[3 * k + r], wh[u][3 * r + q], wl[u][3 * r + q], x_h[q], x_l[q]);
        }
    }
    const int l0 = a.lbeg[c], nl = a.lbeg[c + 1] - l0;
    for (int e0 = lane; e0 < nl; e0 += U * G) {
      float wh[U][9], wl[U][9];
      int cc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * G;
        const int L = l0 + (e < nl ? e : nl - 1);
        const bool in = e < nl && sym3_inside(a, R.qx + a.ld[L][0], R.qy + a.ld[L][1], R.qz + a.ld[L][2]);
        const int cs = a.lcls[L];
        const int jx = R.ix + a.ldel[L][0], jy = R.iy + a.ldel[L][1], jz = R.iz + a.ldel[L][2];
        const int rj = in ? jx + a.pext[cs] * (jy + a.ext[cs][1] * jz) : 0;
        const size_t rcs = (size_t)a.prows[cs];
        const size_t base = a.lbase[L] + rj;
        cc[u] = min(max(R.row + a.llin[L], 0), last);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const float h = vh[base + k * rcs], l = vl[base + k * rcs];
          wh[u][k] = in ? h : 0.f;
          wl[u][k] = in ? l : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          float x_h[3], x_l[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) x_h[q] = xh[(3 * k + q) * xs + cc[u]], x_l[q] = xl[(3 * k + q) * xs + cc[u]];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q)  // transpose of A(j, i)
              df_madd(acc[3 * k + r], wh[u][3 * q + r], wl[u][3 * q + r], x_h[q], x_l[q]);
        }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < 3 * K; ++r) {
      const float oh = __shfl_xor_sync(0xffffffffu, acc[r].h, o);
      const float ol = __shfl_xor_sync(0xffffffffu, acc[r].l, o);
      df_add(acc[r], oh, ol);
    }
  if (R.valid && lane == 0) {
#pragma unroll
    for (int r = 0; r < 3 * K; ++r) {
      const size_t i = r * xs + R.row;
      y[i] = b[i] - ((double)acc[r].h + (double)acc[r].l);
    }
  }
}

// algorithmic bytes: stored values once (the transposed second read is meant
// to be an L2 hit by the launch order), x gathered once, y (and b) once
double sym3_bytes(const Sym3Op& so, int esz, int rows, int streams) {
  return (double)so.total * esz + (double)esz * 3.0 * rows * (1 + streams);
}

template <int G, int U, class T>
static void sym3_launch_g(const Exec& ex, const Csr& m, const T* x, T* y, const T* b, const DotScratch* ds,
                          double* dot) {
  const Sym3Op& so = *m.sym;
  const Sym3Args a = sym3_args(so, G);
  const int nvb = sym3_blocks(so, a);
  if (nvb == 0) return;
  // one resident wave walks the virtual blocks in plane order (measured faster
  // than one block per virtual block: 171 against 200 us at 48^3)
  static thread_local int wave[2] = {};  // resident blocks per variant (dot or not)
  int& w = wave[dot ? 1 : 0];
  if (!w) {
    int dev = 0, sms = 0, occ = 0;
    SK_CUDA(cudaGetDevice(&dev));
    SK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dot) SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sym3<G, U, T, true>, kSymBlock, 0));
    else SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sym3<G, U, T, false>, kSymBlock, 0));
    w = std::max(1, sms * std::max(1, occ));
  }
  const int grid = std::min(nvb, w);
  if (dot) {
    SK_REQUIRE(ds && ds->fused_partial && grid <= ds->fused_cap, STOKES_ERR_ARG, "fused dot scratch too small");
    k_sym3<G, U, T, true><<<grid, kSymBlock, 0, ex.s>>>(a, nvb, so.template v<T>(), x, (size_t)m.rows, b, y,
                                                    ds->fused_partial, ds->fused_counter, dot);
  } else {
    k_sym3<G, U, T, false><<<grid, kSymBlock, 0, ex.s>>>(a, nvb, so.template v<T>(), x, (size_t)m.rows, b, y, nullptr,
                                                     nullptr, nullptr);
  }
  SK_CHECK_LAUNCH();
}

// four right-hand sides (x, y, b: [4][3][rows]): every stored block read once
// for the four; one thread per row, two entries' loads in flight
template <class T> void sym3_launch4(const Exec& ex, const Csr& m, const T* x, T* y, const T* b) {
  const Sym3Op& so = *m.sym;
  const Sym3Args a = sym3_args(so, 1);
  const int nvb = sym3_blocks(so, a);
  if (nvb == 0) return;
  static thread_local int w = 0;
  if (!w) {
    int dev = 0, sms = 0, occ = 0;
    SK_CUDA(cudaGetDevice(&dev));
    SK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sym3<1, 2, T, false, 4>, kSymBlock, 0));
    w = std::max(1, sms * std::max(1, occ));
  }
  const int grid = std::min(nvb, w);
  k_sym3<1, 2, T, false, 4><<<grid, kSymBlock, 0, ex.s>>>(a, nvb, so.template v<T>(), x, (size_t)m.rows, b, y, nullptr,
                                                       nullptr, nullptr);
  SK_CHECK_LAUNCH();
}

template <class T>
void sym3_launch(const Exec& ex, const Csr& m, const T* x, T* y, const T* b, const DotScratch* ds, double* dot) {
  // (threads per row, entries in flight per lane)
  const int g = m.sym->group, u = m.sym->batch;
  if (g == 1 && u == 2) sym3_launch_g<1, 2, T>(ex, m, x, y, b, ds, dot);
  else if (g == 1 && u == 4) sym3_launch_g<1, 4, T>(ex, m, x, y, b, ds, dot);
  else if (g == 1) sym3_launch_g<1, 8, T>(ex, m, x, y, b, ds, dot);
  else if (g == 2 && u == 2) sym3_launch_g<2, 2, T>(ex, m, x, y, b, ds, dot);
  else if (g == 2) sym3_launch_g<2, 4, T>(ex, m, x, y, b, ds, dot);
  else if (g == 4) sym3_launch_g<4, 2, T>(ex, m, x, y, b, ds, dot);
  else sym3_launch_g<8, 1, T>(ex, m, x, y, b, ds, dot);
}

template <int G>
static void sym3_df_g(const Exec& ex, const Csr& m, const float* xh, const float* xl, const double* b, double* y) {
  const Sym3Op& so = *m.sym;
  const Sym3Args a = sym3_args(so, G);
  const int grid = sym3_blocks(so, a);
  if (grid == 0) return;
  k_sym3_df<G><<<grid, kSymBlock, 0, ex.s>>>(a, so.v32, so.v32lo, xh, xl, (size_t)m.rows, b, y);
  SK_CHECK_LAUNCH();
}

// four right-hand sides in one sweep (one thread per row, one entry in flight)
void sym3_residual_df4(const Exec& ex, const Csr& m, const float* xh, const float* xl, const double* b, double* y) {
  const Sym3Op& so = *m.sym;
  const Sym3Args a = sym3_args(so, 1);
  const int grid = sym3_blocks(so, a);
  if (grid == 0) return;
  k_sym3_df<1, 4><<<grid, kSymBlock, 0, ex.s>>>(a, so.v32, so.v32lo, xh, xl, (size_t)m.rows, b, y);
  SK_CHECK_LAUNCH();
}

void sym3_residual_df(const Exec& ex, const Csr& m, const float* xh, const float* xl, const double* b, double* y) {
  switch (m.sym->group) {
    case 1: sym3_df_g<1>(ex, m, xh, xl, b, y); break;
    case 2: sym3_df_g<2>(ex, m, xh, xl, b, y); break;
    case 8: sym3_df_g<8>(ex, m, xh, xl, b, y); break;
    default: sym3_df_g<4>(ex, m, xh, xl, b, y); break;
  }
}

template void sym3_launch<float>(const Exec&, const Csr&, const float*, float*, const float*, const DotScratch*,
                                 double*);
template void sym3_launch4<float>(const Exec&, const Csr&, const float*, float*, const float*);
template void sym3_launch4<double>(const Exec&, const Csr&, const double*, double*, const double*);
template void sym3_launch<double>(const Exec&, const Csr&, const double*, double*, const double*, const DotScratch*,
                                  double*);

}  // namespace sk
