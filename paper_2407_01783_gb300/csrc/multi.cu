// Vector kernels for K right-hand sides solved in lockstep (stokes_solve_multi).
//
// A K-vector holds the reduced unknowns of K systems in two blocks: the
// velocities [K][3][nvi] (so the K x 3 components are one component-major
// set of 3K right-hand sides for the multigrid and stencil products) followed
// by the pressures [K][np]. The "segment" of right-hand side k is its
// velocity part, its pressure part, or both. Every kernel here runs a 2D grid:
// blockIdx.y is the right-hand side, so the K systems keep their own
// coefficients and dot products while sharing one launch. Dot products are
// reduced in a fixed order (deterministic): per-thread sums in FP64 (FP64
// vectors) or double-float (FP32 vectors), FP64 across threads.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace sk {

struct KSeg {
  size_t nu, np;  // velocity / pressure entries per right-hand side
  int K;
  int parts;      // 1: velocity, 2: pressure, 3: both
  __device__ __forceinline__ size_t len() const { return (parts & 1 ? nu : 0) + (parts & 2 ? np : 0); }
  // address of entry e of right-hand side k's segment in a K-vector
  __device__ __forceinline__ size_t at(int k, size_t e) const {
    if (parts & 1) {
      if (e < nu) return (size_t)k * nu + e;
      e -= nu;
    }
    return (size_t)K * nu + (size_t)k * np + e;
  }
};

// Per-thread sums: FP64 for FP64 vectors; for FP32 vectors double-float
// (df_dot) on the FP32 units, since FP64 arithmetic is scarce on this GPU and
// would bound these kernels before memory does. Across threads: FP64.
template <class T>
__global__ void __launch_bounds__(256) k_kdot(KSeg s, const T* __restrict__ x, const T* __restrict__ y,
                                              double* partial, unsigned* counter, double* out) {
  const int k = blockIdx.y;
  const size_t n = s.len();
  double t = 0.0;
  if constexpr (std::is_same<T, float>::value) {
    DF a{0.f, 0.f};
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
      const size_t i = s.at(k, e);
      df_dot(a, x[i], y ? y[i] : 1.f);
    }
    t = (double)a.h + (double)a.l;
  } else {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
      const size_t i = s.at(k, e);
      t += (double)x[i] * (y ? (double)y[i] : 1.0);
    }
  }
  grid_sum(t, partial + (size_t)k * gridDim.x, counter + k, out + k);
}

// y_k = a_k x_k + b_k y_k on the chosen segment (x may alias y)
template <class T>
__global__ void __launch_bounds__(256) k_kaxpby(KSeg s, KCoefs a, const T* x, KCoefs b, T* y, int* flag) {
  const int k = blockIdx.y;
  __shared__ double ab[2];
  if (threadIdx.x == 0) {
    ab[0] = a.value(k, blockIdx.x == 0 ? flag : nullptr);
    ab[1] = b.value(k, blockIdx.x == 0 ? flag : nullptr);
  }
  __syncthreads();
  const T av = (T)ab[0], bv = (T)ab[1];
  const size_t n = s.len();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = s.at(k, e);
    y[i] = bv == T(0) ? av * x[i] : av * x[i] + bv * y[i];
  }
}

// y_k += c_k (a constant per right-hand side, c_k = scale * num_k / den_k)
template <class T>
__global__ void __launch_bounds__(256) k_kaddconst(KSeg s, KCoefs c, T* y, int* flag) {
  const int k = blockIdx.y;
  __shared__ double cv;
  if (threadIdx.x == 0) cv = c.value(k, blockIdx.x == 0 ? flag : nullptr);
  __syncthreads();
  const T v = (T)cv;
  const size_t n = s.len();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[s.at(k, e)] += v;
}

// out[k * ld + i] = V_i(k) . w(k) for i < J <= KB: w read once; per right-hand
// side the partials of all J sums in block order, reduced by the last block
template <class T, int KB>
__global__ void __launch_bounds__(256) k_kmdot(KSeg s, KBasis<T> V, int J, const T* __restrict__ w, double* partial,
                                               unsigned* counter, double* out, int ld) {
  const int k = blockIdx.y;
  const size_t n = s.len();
  double acc[KB];
  if constexpr (std::is_same<T, float>::value) {  // double-float per thread, as k_kdot
    DF a[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) a[i] = DF{0.f, 0.f};
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
      const size_t q = s.at(k, e);
      const float we = w[q];
#pragma unroll
      for (int i = 0; i < KB; ++i)
        if (i < J) df_dot(a[i], V.v[i][q], we);
    }
#pragma unroll
    for (int i = 0; i < KB; ++i) acc[i] = (double)a[i].h + (double)a[i].l;
  } else {
#pragma unroll
    for (int i = 0; i < KB; ++i) acc[i] = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
      const size_t a = s.at(k, e);
      const double we = (double)w[a];
#pragma unroll
      for (int i = 0; i < KB; ++i)
        if (i < J) acc[i] += (double)V.v[i][a] * we;
    }
  }
  __shared__ double sh[8][KB];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < KB; ++i) {
    double v = acc[i];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][i] = v;
  }
  __syncthreads();
  double* part = partial + (size_t)k * KB * gridDim.x;
  if (threadIdx.x < J) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += sh[q][threadIdx.x];
    part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter + k, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = wid; i < J; i += (int)(blockDim.x >> 5)) {
    double v = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) v += __ldcg(&part[(size_t)i * gridDim.x + b]);
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[(size_t)k * ld + i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) counter[k] = 0u;
}

// w(k) += sign * sum_{i < J} h_ki V_i(k), h_ki = h[k * ld + i] (device) or hc.c[k * ld + i]
template <class T, int KB>
__global__ void __launch_bounds__(256) k_kmaxpy(KSeg s, KBasis<T> V, int J, const double* h, KHost hc, int ld,
                                                double sign, T* w) {
  const int k = blockIdx.y;
  __shared__ T c[KB];
  if (threadIdx.x < KB)
    c[threadIdx.x] =
        (int)threadIdx.x < J ? (T)(sign * (h ? h[(size_t)k * ld + threadIdx.x] : hc.c[k * ld + threadIdx.x])) : T(0);
  __syncthreads();
  const size_t n = s.len();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t a = s.at(k, e);
    T acc = w[a];
#pragma unroll
    for (int i = 0; i < KB; ++i)
      if (i < J) acc += c[i] * V.v[i][a];
    w[a] = acc;
  }
}

__global__ void k_ksub(int K, double* out, const double* a, const double* b) {
  const int k = threadIdx.x;
  if (k < K) out[k] = a[k] - b[k];
}

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
constexpr int kKGridMax = 2 * 152;  // blocks per right-hand side
static KSeg kseg(size_t nu, size_t np, int K, int parts) { return KSeg{nu, np, K, parts}; }
static size_t seglen(size_t nu, size_t np, int parts) { return (parts & 1 ? nu : 0) + (parts & 2 ? np : 0); }
static int kgrid(size_t len) {
  return (int)std::max<long long>(1, std::min<long long>(cdiv((long long)len, 256), kKGridMax));
}
static int pow2_ge(int k) {
  int K = 1;
  while (K < k) K <<= 1;
  return K;
}

long long kdot_scratch(size_t len_max, int K) { return (long long)kgrid(len_max) * K * kMaxBasisK; }

template <class T>
void kdot(const Exec& ex, const DotScratch& ds, size_t nu, size_t np, int K, int parts, const T* x, const T* y,
          double* out) {
  const size_t len = seglen(nu, np, parts);
  const int gx = kgrid(len);
  SK_REQUIRE(K >= 1 && K <= kMaxRhs, STOKES_ERR_ARG, "kdot: 1 to 8 right-hand sides");
  SK_REQUIRE(ds.k_partial && (long long)gx * K <= ds.k_cap, STOKES_ERR_ARG, "kdot: scratch too small");
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * K * len * (y ? 2.0 : 1.0));
  k_kdot<T><<<dim3(gx, K), 256, 0, ex.s>>>(kseg(nu, np, K, parts), x, y, ds.k_partial, ds.k_counter, out);
  SK_CHECK_LAUNCH();
}

template <class T>
void kaxpby(const Exec& ex, size_t nu, size_t np, int K, int parts, const KCoefs& a, const T* x, const KCoefs& b,
            T* y) {
  SK_REQUIRE(K >= 1 && K <= kMaxRhs, STOKES_ERR_ARG, "kaxpby: 1 to 8 right-hand sides");
  const size_t len = seglen(nu, np, parts);
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * K * len * 3.0);
  k_kaxpby<T><<<dim3(kgrid(len), K), 256, 0, ex.s>>>(kseg(nu, np, K, parts), a, x, b, y, ex.flag);
  SK_CHECK_LAUNCH();
}

template <class T>
void kaddconst(const Exec& ex, size_t nu, size_t np, int K, int parts, const KCoefs& c, T* y) {
  SK_REQUIRE(K >= 1 && K <= kMaxRhs, STOKES_ERR_ARG, "kaddconst: 1 to 8 right-hand sides");
  const size_t len = seglen(nu, np, parts);
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * K * len * 2.0);
  k_kaddconst<T><<<dim3(kgrid(len), K), 256, 0, ex.s>>>(kseg(nu, np, K, parts), c, y, ex.flag);
  SK_CHECK_LAUNCH();
}

template <class T>
void kmdot(const Exec& ex, const DotScratch& ds, size_t nu, size_t np, int K, int J, const T* const* V, const T* w,
           double* out, int ld) {
  SK_REQUIRE(J >= 1 && J <= kMaxBasisK && K >= 1 && K <= kMaxRhs, STOKES_ERR_ARG, "kmdot: bad count");
  const size_t len = seglen(nu, np, 3);
  const int gx = kgrid(len);
  const int KB = pow2_ge(J);
  SK_REQUIRE(ds.k_partial && (long long)gx * K * KB <= ds.k_cap, STOKES_ERR_ARG, "kmdot: scratch too small");
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * K * len * (J + 1.0));
  KBasis<T> B{};
  for (int i = 0; i < J; ++i) B.v[i] = V[i];
  const KSeg sg = kseg(nu, np, K, 3);
  const dim3 grid(gx, K);
  switch (KB) {
    case 1: k_kmdot<T, 1><<<grid, 256, 0, ex.s>>>(sg, B, J, w, ds.k_partial, ds.k_counter, out, ld); break;
    case 2: k_kmdot<T, 2><<<grid, 256, 0, ex.s>>>(sg, B, J, w, ds.k_partial, ds.k_counter, out, ld); break;
    case 4: k_kmdot<T, 4><<<grid, 256, 0, ex.s>>>(sg, B, J, w, ds.k_partial, ds.k_counter, out, ld); break;
    case 8: k_kmdot<T, 8><<<grid, 256, 0, ex.s>>>(sg, B, J, w, ds.k_partial, ds.k_counter, out, ld); break;
    case 16: k_kmdot<T, 16><<<grid, 256, 0, ex.s>>>(sg, B, J, w, ds.k_partial, ds.k_counter, out, ld); break;
    default: k_kmdot<T, 32><<<grid, 256, 0, ex.s>>>(sg, B, J, w, ds.k_partial, ds.k_counter, out, ld); break;
  }
  SK_CHECK_LAUNCH();
}

template <class T>
void kmaxpy(const Exec& ex, size_t nu, size_t np, int K, int J, const T* const* V, const double* h,
            const double* hhost, int ld, double sign, T* w) {
  SK_REQUIRE(J >= 1 && J <= kMaxBasisK && K >= 1 && K <= kMaxRhs, STOKES_ERR_ARG, "kmaxpy: bad count");
  SK_REQUIRE(!hhost || (long long)K * ld <= kMaxRhs * kMaxBasisK, STOKES_ERR_ARG, "kmaxpy: too many coefficients");
  const size_t len = seglen(nu, np, 3);
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * K * len * (J + 2.0));
  KBasis<T> B{};
  for (int i = 0; i < J; ++i) B.v[i] = V[i];
  KHost hc{};
  if (hhost)
    for (int k = 0; k < K; ++k)
      for (int i = 0; i < J; ++i) hc.c[k * ld + i] = hhost[k * ld + i];
  const KSeg sg = kseg(nu, np, K, 3);
  const dim3 grid(kgrid(len), K);
  switch (pow2_ge(J)) {
    case 1: k_kmaxpy<T, 1><<<grid, 256, 0, ex.s>>>(sg, B, J, h, hc, ld, sign, w); break;
    case 2: k_kmaxpy<T, 2><<<grid, 256, 0, ex.s>>>(sg, B, J, h, hc, ld, sign, w); break;
    case 4: k_kmaxpy<T, 4><<<grid, 256, 0, ex.s>>>(sg, B, J, h, hc, ld, sign, w); break;
    case 8: k_kmaxpy<T, 8><<<grid, 256, 0, ex.s>>>(sg, B, J, h, hc, ld, sign, w); break;
    case 16: k_kmaxpy<T, 16><<<grid, 256, 0, ex.s>>>(sg, B, J, h, hc, ld, sign, w); break;
    default: k_kmaxpy<T, 32><<<grid, 256, 0, ex.s>>>(sg, B, J, h, hc, ld, sign, w); break;
  }
  SK_CHECK_LAUNCH();
}

void ksub(const Exec& ex, int K, double* out, const double* a, const double* b) {
  SK_REQUIRE(K >= 1 && K <= kMaxRhs, STOKES_ERR_ARG, "ksub: 1 to 8 values");
  ProfScope ps(ex, STOKES_KERNEL_OTHER, 24.0 * K);
  k_ksub<<<1, 32, 0, ex.s>>>(K, out, a, b);
  SK_CHECK_LAUNCH();
}

#define SK_INSTK(T)                                                                                                  \
  template void kdot<T>(const Exec&, const DotScratch&, size_t, size_t, int, int, const T*, const T*, double*);     \
  template void kaxpby<T>(const Exec&, size_t, size_t, int, int, const KCoefs&, const T*, const KCoefs&, T*);      \
  template void kaddconst<T>(const Exec&, size_t, size_t, int, int, const KCoefs&, T*);                           \
  template void kmdot<T>(const Exec&, const DotScratch&, size_t, size_t, int, int, const T* const*, const T*,      \
                         double*, int);                                                                              \
  template void kmaxpy<T>(const Exec&, size_t, size_t, int, int, const T* const*, const double*, const double*, int, \
                          double, T*);
SK_INSTK(float)
SK_INSTK(double)

}  // namespace sk
