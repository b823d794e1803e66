// Vector kernels for the Krylov solvers: multi-dot products accumulated in
// FP64 with a fixed reduction order (per-block partials, then the last block
// to finish sums them in block order), and fused axpy-type updates whose
// coefficients are read from device-resident scalars so that the host never
// waits for a dot product it does not need to see.
#include <cmath>

#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace sk {

__device__ __forceinline__ double coef_value(const Coef& k, int* flag) {
  double v = k.c;
  if (k.num) {
    const double den = k.den ? *k.den : 1.0;
    if (k.positive && !(den > 0.0)) {
      // r^T z <= 0 in a preconditioned CG: an indefinite preconditioner, or
      // vanished Krylov vectors (exact convergence inside a fixed-iteration
      // solve). Flag it (the host reports a breakdown only if the solve then
      // fails) and contribute nothing.
      if (flag) atomicOr(flag, 1);
      return v;
    }
    // a zero denominator only arises when the Krylov vectors vanished (exact
    // convergence inside a fixed-iteration solve): contribute nothing
    if (den != 0.0) v += k.s * (*k.num) / den;
  }
  return v;
}

template <class T> struct DotArgs {
  const T* x[kMaxDots];
  const T* y[kMaxDots];
  int k;
  int compensated;  // FP32 inputs: per-thread Neumaier sums in FP32, FP64 across threads
  size_t n;
  double* partial;
  unsigned* counter;
  double* out;
};

template <class T, int K>
__global__ void __launch_bounds__(256) k_dots(DotArgs<T> a) {
  double s[K];
#pragma unroll
  for (int j = 0; j < K; ++j) s[j] = 0.0;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  if (a.compensated) {
    // GB300 runs FP64 at a small fraction of its FP32 rate, so products and
    // per-thread sums of FP32 vectors stay in FP32 with Neumaier's compensated
    // summation (error ~ eps_32 per product, not per partial sum); only the
    // cross-thread reduction is FP64.
    // four independent accumulators per dot keep four loads per vector in
    // flight per thread
    float fs[K][4], fc[K][4];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
      for (int u = 0; u < 4; ++u) fs[j][u] = 0.f, fc[j][u] = 0.f;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < a.n; i += 4 * stride) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        float p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = (float)a.x[j][i + u * stride] * (a.y[j] ? (float)a.y[j][i + u * stride] : 1.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float t = fs[j][u] + p[u];
          fc[j][u] += fabsf(fs[j][u]) >= fabsf(p[u]) ? (fs[j][u] - t) + p[u] : (p[u] - t) + fs[j][u];
          fs[j][u] = t;
        }
      }
    }
    for (; i < a.n; i += stride) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const float p = (float)a.x[j][i] * (a.y[j] ? (float)a.y[j][i] : 1.f);
        const float t = fs[j][0] + p;
        fc[j][0] += fabsf(fs[j][0]) >= fabsf(p) ? (fs[j][0] - t) + p : (p - t) + fs[j][0];
        fs[j][0] = t;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
      for (int u = 0; u < 4; ++u) s[j] += (double)fs[j][u] + (double)fc[j][u];
  } else {
    double t[K][4];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
      for (int u = 0; u < 4; ++u) t[j][u] = 0.0;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < a.n; i += 4 * stride) {
#pragma unroll
      for (int j = 0; j < K; ++j)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          t[j][u] += (double)a.x[j][i + u * stride] * (a.y[j] ? (double)a.y[j][i + u * stride] : 1.0);
    }
    for (; i < a.n; i += stride) {
#pragma unroll
      for (int j = 0; j < K; ++j) t[j][0] += (double)a.x[j][i] * (a.y[j] ? (double)a.y[j][i] : 1.0);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) s[j] = (t[j][0] + t[j][1]) + (t[j][2] + t[j][3]);
  }
  __shared__ double sh[K][8];
  __shared__ bool last;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double v = s[j];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[j][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    a.partial[threadIdx.x * gridDim.x + blockIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  // the last block: fixed-order sum of the partials
  for (int j = 0; j < K; ++j) {
    double v = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(&a.partial[j * gridDim.x + b]);
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[0][wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[0][w];
      a.out[j] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.counter = 0u;
}

template <class T>
void dots(const Exec& ex, const DotScratch& ds, int k, const T* const* x, const T* const* y, size_t n, double* out,
          int mode) {
  SK_REQUIRE(k >= 1 && k <= kMaxDots, STOKES_ERR_ARG, "dots: bad count");
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, 0.0 + (double)sizeof(T) * n * (2.0 * k));
  DotArgs<T> a{};
  for (int j = 0; j < k; ++j) a.x[j] = x[j], a.y[j] = y ? y[j] : nullptr;
  a.k = k;
  a.n = n;
  a.compensated = std::is_same<T, float>::value &&
                  (mode == kDotFast || (mode == kDotAuto && n >= kCompensatedMin));
  a.partial = ds.partial;
  a.counter = ds.counter;
  a.out = out;
  int grid = (int)std::min<long long>(kDotBlocks, std::max<long long>(1, cdiv((long long)n, 256)));
  switch (k) {
    case 1: k_dots<T, 1><<<grid, 256, 0, ex.s>>>(a); break;
    case 2: k_dots<T, 2><<<grid, 256, 0, ex.s>>>(a); break;
    case 3: k_dots<T, 3><<<grid, 256, 0, ex.s>>>(a); break;
    default: k_dots<T, 4><<<grid, 256, 0, ex.s>>>(a); break;
  }
  SK_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Multi-vector kernels for the Arnoldi process (classical Gram-Schmidt):
// out[i] = V_i . w for up to kMaxBasis vectors in one pass that reads w once,
// and w -= sum_i h_i V_i in one pass. FP64 accumulation in a fixed order.
// ---------------------------------------------------------------------------
template <class T> struct MultiArgs {
  const T* v[kMaxBasis];
  double c[kMaxBasis];     // host coefficients (when dev == nullptr)
  const double* dev;       // device coefficients h[0..k-1], or null
  int k;
  double sign;
  size_t n;
  T* w;
  const T* wr;             // w for the dot kernel
  double* partial;         // [k][gridDim.x]
  unsigned* counter;
  double* out;
};

// K: the compile-time bound (a power of two >= a.k), so the basis pointers and
// accumulators are indexed statically
template <class T, int K>
__global__ void __launch_bounds__(256) k_mdot(MultiArgs<T> a) {
  double s[K];
  if constexpr (std::is_same<T, float>::value) {
    // FP32 vectors: per-thread double-float sums (df_dot) on the FP32 units
    // (FP64 arithmetic would bound the kernel before memory does)
    DF d[K];
#pragma unroll
    for (int i = 0; i < K; ++i) d[i] = DF{0.f, 0.f};
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.n; e += (size_t)gridDim.x * blockDim.x) {
      const float we = a.wr[e];
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i < a.k) df_dot(d[i], a.v[i][e], we);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) s[i] = (double)d[i].h + (double)d[i].l;
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) s[i] = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.n; e += (size_t)gridDim.x * blockDim.x) {
      const double we = (double)a.wr[e];
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i < a.k) s[i] += (double)a.v[i][e] * we;
    }
  }
  __shared__ double sh[8][K];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double v = s[i];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < a.k) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
    a.partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block: for each vector, the partials in block order (one warp per vector)
  for (int i = wid; i < a.k; i += (int)(blockDim.x >> 5)) {
    double v = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) v += __ldcg(&a.partial[(size_t)i * gridDim.x + b]);
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) a.out[i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) *a.counter = 0u;
}

template <class T, int K>
__global__ void __launch_bounds__(256) k_maxpy(MultiArgs<T> a) {
  __shared__ T h[K];
  if (threadIdx.x < K) h[threadIdx.x] = threadIdx.x < a.k ? (T)(a.sign * (a.dev ? a.dev[threadIdx.x] : a.c[threadIdx.x])) : T(0);
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.n; e += (size_t)gridDim.x * blockDim.x) {
    T acc = a.w[e];
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i < a.k) acc += h[i] * a.v[i][e];
    a.w[e] = acc;
  }
}

static inline int pow2_at_least(int k) {
  int K = 1;
  while (K < k) K <<= 1;
  return K;
}

template <class T>
void mdot(const Exec& ex, const DotScratch& ds, int k, const T* const* V, const T* w, size_t n, double* out) {
  SK_REQUIRE(k >= 1 && k <= kMaxBasis, STOKES_ERR_ARG, "mdot: bad count");
  const int grid = (int)std::min<long long>(kDotBlocks, std::max<long long>(1, cdiv((long long)n, 256)));
  SK_REQUIRE(ds.fused_partial && (long long)grid * k <= ds.fused_cap, STOKES_ERR_ARG, "mdot: scratch too small");
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * (k + 1.0));
  MultiArgs<T> a{};
  for (int i = 0; i < k; ++i) a.v[i] = V[i];
  a.k = k;
  a.n = n;
  a.wr = w;
  a.partial = ds.fused_partial;
  a.counter = ds.fused_counter;
  a.out = out;
  switch (pow2_at_least(k)) {
    case 1: k_mdot<T, 1><<<grid, 256, 0, ex.s>>>(a); break;
    case 2: k_mdot<T, 2><<<grid, 256, 0, ex.s>>>(a); break;
    case 4: k_mdot<T, 4><<<grid, 256, 0, ex.s>>>(a); break;
    case 8: k_mdot<T, 8><<<grid, 256, 0, ex.s>>>(a); break;
    case 16: k_mdot<T, 16><<<grid, 256, 0, ex.s>>>(a); break;
    default: k_mdot<T, 32><<<grid, 256, 0, ex.s>>>(a); break;
  }
  SK_CHECK_LAUNCH();
}

template <class T>
void maxpy(const Exec& ex, int k, const double* dev_coef, const double* host_coef, double sign, const T* const* V,
           T* w, size_t n) {
  SK_REQUIRE(k >= 1 && k <= kMaxBasis, STOKES_ERR_ARG, "maxpy: bad count");
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * (k + 2.0));
  MultiArgs<T> a{};
  for (int i = 0; i < k; ++i) {
    a.v[i] = V[i];
    a.c[i] = host_coef ? host_coef[i] : 0.0;
  }
  a.dev = dev_coef;
  a.k = k;
  a.sign = sign;
  a.n = n;
  a.w = w;
  const int grid = (int)std::min<long long>(cdiv((long long)n, 256), 8 * 152);  // as the elementwise kernels
  switch (pow2_at_least(k)) {
    case 1: k_maxpy<T, 1><<<grid, 256, 0, ex.s>>>(a); break;
    case 2: k_maxpy<T, 2><<<grid, 256, 0, ex.s>>>(a); break;
    case 4: k_maxpy<T, 4><<<grid, 256, 0, ex.s>>>(a); break;
    case 8: k_maxpy<T, 8><<<grid, 256, 0, ex.s>>>(a); break;
    case 16: k_maxpy<T, 16><<<grid, 256, 0, ex.s>>>(a); break;
    default: k_maxpy<T, 32><<<grid, 256, 0, ex.s>>>(a); break;
  }
  SK_CHECK_LAUNCH();
}

// Elementwise kernels run a grid-stride loop over at most kEwBlocks blocks
// (8 resident 256-thread blocks per SM): a block's coefficient prologue is paid
// once per ~8 elements per thread rather than once per 256 elements.
constexpr int kEwBlocks = 8 * 152;
static inline int ew_grid(size_t n) { return (int)std::min<long long>(cdiv((long long)n, 256), kEwBlocks); }
#define SK_GRID(n) ew_grid(n), 256, 0, ex.s
#define SK_LOOP(i) \
  _Pragma("unroll 4") for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)

// Coefficients from device scalars are evaluated once per block (one FP64
// division per block instead of per element: GB300's FP64 rate is low).
#define SK_COEF2(A, B, va, vb)                                  \
  __shared__ double sk_coef_[2];                                \
  if (threadIdx.x == 0) {                                       \
    sk_coef_[0] = coef_value(A, blockIdx.x == 0 ? flag : nullptr); \
    sk_coef_[1] = coef_value(B, blockIdx.x == 0 ? flag : nullptr); \
  }                                                             \
  __syncthreads();                                              \
  const double va = sk_coef_[0], vb = sk_coef_[1];

template <class T>
__global__ void k_axpby(size_t n, Coef a, const T* __restrict__ x, Coef b, T* __restrict__ y, int* flag) {
  SK_COEF2(a, b, ad, bd);
  const T av = (T)ad, bv = (T)bd;
  if (bv == T(0)) {
    SK_LOOP(i) { y[i] = av * x[i]; }
  } else {
    SK_LOOP(i) { y[i] = av * x[i] + bv * y[i]; }
  }
}
template <class T> void axpby(const Exec& ex, size_t n, Coef a, const T* x, Coef b, T* y) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * 3);
  k_axpby<T><<<SK_GRID(n)>>>(n, a, x, b, y, ex.flag);
  SK_CHECK_LAUNCH();
}

template <class T>
__global__ void k_cg_update(size_t n, Coef a, const T* __restrict__ d, T* __restrict__ x, const T* __restrict__ q,
                            T* __restrict__ r, int* flag) {
  SK_COEF2(a, a, ad, unused);
  (void)unused;
  if (blockIdx.x == 0 && threadIdx.x == 0 && flag && a.den && !(*a.den > 0.0))
    atomicOr(flag, 1);  // p^T A p <= 0: breakdown
  const T av = (T)ad;
  if (r) {
    SK_LOOP(i) {
      x[i] += av * d[i];
      r[i] -= av * q[i];
    }
  } else {
    SK_LOOP(i) { x[i] += av * d[i]; }
  }
}
template <class T> void cg_update(const Exec& ex, size_t n, Coef a, const T* d, T* x, const T* q, T* r) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * (r ? 6 : 3));
  k_cg_update<T><<<SK_GRID(n)>>>(n, a, d, x, q, r, ex.flag);
  SK_CHECK_LAUNCH();
}

// x += a d; r -= a q; *rr = r . r (new r), the squares summed per thread in
// FP64 and over the grid in a fixed order (grid_sum)
template <class T>
__global__ void k_cg_update_rr(size_t n, Coef a, const T* __restrict__ d, T* __restrict__ x, const T* __restrict__ q,
                               T* __restrict__ r, int* flag, double* partial, unsigned* counter, double* rr) {
  SK_COEF2(a, a, ad, unused);
  (void)unused;
  if (blockIdx.x == 0 && threadIdx.x == 0 && flag && a.den && !(*a.den > 0.0))
    atomicOr(flag, 1);  // p^T A p <= 0: breakdown
  const T av = (T)ad;
  double s = 0.0;
  SK_LOOP(i) {
    x[i] += av * d[i];
    const T rn = r[i] - av * q[i];
    r[i] = rn;
    s += (double)(rn * rn);
  }
  grid_sum(s, partial, counter, rr);
}
template <class T>
void cg_update_rr(const Exec& ex, const DotScratch& ds, size_t n, Coef a, const T* d, T* x, const T* q, T* r,
                  double* rr) {
  SK_REQUIRE(n > 0, STOKES_ERR_ARG, "cg_update_rr: empty vector");
  const int grid = ew_grid(n);
  SK_REQUIRE(ds.fused_partial && grid <= ds.fused_cap, STOKES_ERR_ARG, "fused dot scratch too small");
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * 6);
  k_cg_update_rr<T><<<grid, 256, 0, ex.s>>>(n, a, d, x, q, r, ex.flag, ds.fused_partial, ds.fused_counter, rr);
  SK_CHECK_LAUNCH();
}

template <class T>
__global__ void k_scale_copy(size_t n, Coef a, const T* __restrict__ x, T* __restrict__ y, int* flag) {
  SK_COEF2(a, a, ad, unused);
  (void)unused;
  SK_LOOP(i) {
    y[i] = (T)ad * x[i];
  }
}
template <class T> void scale_copy(const Exec& ex, size_t n, Coef a, const T* x, T* y) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * 2);
  k_scale_copy<T><<<SK_GRID(n)>>>(n, a, x, y, ex.flag);
  SK_CHECK_LAUNCH();
}

template <class T>
__global__ void k_lincomb2(size_t n, T c1, const T* __restrict__ x1, T c2, const T* __restrict__ x2, T* __restrict__ y) {
  SK_LOOP(i) {
    y[i] = c1 * x1[i] + c2 * x2[i];
  }
}
template <class T> void lincomb2(const Exec& ex, size_t n, double c1, const T* x1, double c2, const T* x2, T* y) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * 3);
  k_lincomb2<T><<<SK_GRID(n)>>>(n, (T)c1, x1, (T)c2, x2, y);
  SK_CHECK_LAUNCH();
}

template <class T> __global__ void k_sub_ratio(size_t n, const double* num, const double* den, double scale, T* x) {
  __shared__ double sk_v;
  if (threadIdx.x == 0) sk_v = scale * (*num) / (den ? *den : 1.0);
  __syncthreads();
  SK_LOOP(i) {
    x[i] -= (T)sk_v;
  }
}
template <class T> void sub_mean(const Exec& ex, size_t n, const double* sum, double count, T* r) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * 2);
  k_sub_ratio<T><<<SK_GRID(n)>>>(n, sum, nullptr, 1.0 / count, r);
  SK_CHECK_LAUNCH();
}
template <class T> void sub_ratio(const Exec& ex, size_t n, const double* num, const double* den, T* x) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * n * 2);
  k_sub_ratio<T><<<SK_GRID(n)>>>(n, num, den, 1.0, x);
  SK_CHECK_LAUNCH();
}

template <class T>
__global__ void k_cheb_first(size_t n, const T* __restrict__ dinv, const T* __restrict__ b, T c,
                             T* __restrict__ d, T* __restrict__ x) {
  // component-major: blockIdx.y is the component, n the rows of one component
  const size_t off = (size_t)blockIdx.y * n;
  SK_LOOP(i) {
    const T v = c * dinv[i] * b[off + i];
    d[off + i] = v;
    x[off + i] = v;
  }
}
template <class T> void cheb_first(const Exec& ex, size_t n, int nr, const T* dinv, const T* b, double c, T* d, T* x) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * (n * 3 + n / nr));
  const size_t rows = n / nr;
  k_cheb_first<T><<<dim3(std::max(1, ew_grid(rows) / nr), nr), 256, 0, ex.s>>>(rows, dinv, b, (T)c, d, x);
  SK_CHECK_LAUNCH();
}

// node-interleaved vectors: row i's nr values at i * nr (one thread per row)
template <class T, int NR>
__global__ void k_cheb_first_il(size_t n, const T* __restrict__ dinv, const T* __restrict__ b, T c,
                                T* __restrict__ d, T* __restrict__ x) {
  SK_LOOP(i) {
    const T s = c * dinv[i];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const T v = s * b[i * NR + r];
      d[i * NR + r] = v;
      x[i * NR + r] = v;
    }
  }
}
template <class T>
void cheb_first_il(const Exec& ex, size_t n, int nr, const T* dinv, const T* b, double c, T* d, T* x) {
  if (!n) return;
  SK_REQUIRE(nr == 4 || nr == 12, STOKES_ERR_ARG, "interleaved vectors need 4 or 12 components");
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)sizeof(T) * (n * 3 + n / nr));
  const size_t rows = n / nr;
  if (nr == 4) k_cheb_first_il<T, 4><<<SK_GRID(rows)>>>(rows, dinv, b, (T)c, d, x);
  else k_cheb_first_il<T, 12><<<SK_GRID(rows)>>>(rows, dinv, b, (T)c, d, x);
  SK_CHECK_LAUNCH();
}

// [nr][rows] <-> [rows][nr]: a thread per row reads its nr components (each
// read coalesced across the warp) and writes them contiguously, or back
template <class T, int NR, bool TO_IL>
__global__ void k_relayout(size_t n, const T* __restrict__ src, T* __restrict__ dst) {
  // n rows
  SK_LOOP(i) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (TO_IL) dst[i * NR + r] = src[r * n + i];
      else dst[r * n + i] = src[i * NR + r];
    }
  }
}
template <class T> void to_interleaved(const Exec& ex, size_t rows, int nr, const T* cm, T* il) {
  if (!rows) return;
  SK_REQUIRE(nr == 4 || nr == 12, STOKES_ERR_ARG, "interleaved vectors need 4 or 12 components");
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, 2.0 * sizeof(T) * rows * nr);
  if (nr == 4) k_relayout<T, 4, true><<<SK_GRID(rows)>>>(rows, cm, il);
  else k_relayout<T, 12, true><<<SK_GRID(rows)>>>(rows, cm, il);
  SK_CHECK_LAUNCH();
}
template <class T> void to_component_major(const Exec& ex, size_t rows, int nr, const T* il, T* cm) {
  if (!rows) return;
  SK_REQUIRE(nr == 4 || nr == 12, STOKES_ERR_ARG, "interleaved vectors need 4 or 12 components");
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, 2.0 * sizeof(T) * rows * nr);
  if (nr == 4) k_relayout<T, 4, false><<<SK_GRID(rows)>>>(rows, il, cm);
  else k_relayout<T, 12, false><<<SK_GRID(rows)>>>(rows, il, cm);
  SK_CHECK_LAUNCH();
}

// natural <-> parity-split numbering (SplitMap), component-major [nr][rows]
// or, with IL, between natural component-major and split interleaved
// [rows][nr]; a thread per natural row i
template <class T, int NR, bool IL, bool TO>
__global__ void k_split(size_t n, SplitMap sm, const T* __restrict__ src, T* __restrict__ dst) {
  SK_LOOP(i) {
    const size_t j = (size_t)sm((int)i);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const size_t nat = r * n + i;
      const size_t spl = IL ? j * NR + r : r * n + j;
      if (TO) dst[spl] = src[nat];
      else dst[nat] = src[spl];
    }
  }
}
template <class T, bool TO>
static void split_launch(const Exec& ex, size_t rows, int nr, const T* src, T* dst, bool il, const SplitMap& sm) {
  if (!rows) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, 2.0 * sizeof(T) * rows * nr);
  if (il) {
    SK_REQUIRE(nr == 4 || nr == 12, STOKES_ERR_ARG, "interleaved vectors need 4 or 12 components");
    if (nr == 4) k_split<T, 4, true, TO><<<SK_GRID(rows)>>>(rows, sm, src, dst);
    else k_split<T, 12, true, TO><<<SK_GRID(rows)>>>(rows, sm, src, dst);
  } else {
    SK_REQUIRE(nr == 1 || nr == 3, STOKES_ERR_ARG, "split numbering: 1 or 3 components (component-major)");
    if (nr == 1) k_split<T, 1, false, TO><<<SK_GRID(rows)>>>(rows, sm, src, dst);
    else k_split<T, 3, false, TO><<<SK_GRID(rows)>>>(rows, sm, src, dst);
  }
  SK_CHECK_LAUNCH();
}
template <class T> void to_split(const Exec& ex, size_t rows, int nr, const T* src, T* dst, bool il, const SplitMap& sm) {
  split_launch<T, true>(ex, rows, nr, src, dst, il, sm);
}
template <class T>
void from_split(const Exec& ex, size_t rows, int nr, const T* src, T* dst, bool il, const SplitMap& sm) {
  split_launch<T, false>(ex, rows, nr, src, dst, il, sm);
}

template <class S, class D> __global__ void k_convert(size_t n, const S* __restrict__ x, D* __restrict__ y) {
  SK_LOOP(i) {
    y[i] = (D)x[i];
  }
}
template <class S, class D> void convert(const Exec& ex, size_t n, const S* x, D* y) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)(sizeof(S) + sizeof(D)) * n);
  k_convert<S, D><<<SK_GRID(n)>>>(n, x, y);
  SK_CHECK_LAUNCH();
}
template <class S, class D> __global__ void k_add_convert(size_t n, const S* __restrict__ x, D* __restrict__ y) {
  SK_LOOP(i) {
    y[i] += (D)x[i];
  }
}
template <class S, class D> void add_convert(const Exec& ex, size_t n, const S* x, D* y) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, (double)(sizeof(S) + 2 * sizeof(D)) * n);
  k_add_convert<S, D><<<SK_GRID(n)>>>(n, x, y);
  SK_CHECK_LAUNCH();
}

// reduced interior velocity [(2n-1)^3][3] <-> all-node field [(2n+1)^3][3]
__global__ void k_expand(int n, const double* __restrict__ ured, double* __restrict__ uall) {
  int N = 2 * n + 1, m = 2 * n - 1;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)N * N * N;
  if (i >= tot) return;
  int qx = (int)(i % N), qy = (int)((i / N) % N), qz = (int)(i / ((size_t)N * N));
  bool in = qx > 0 && qx < N - 1 && qy > 0 && qy < N - 1 && qz > 0 && qz < N - 1;
  size_t r = in ? (size_t)(qx - 1) + (size_t)m * ((qy - 1) + (size_t)m * (qz - 1)) : 0;
  const size_t nvi = (size_t)m * m * m;
  for (int c = 0; c < 3; ++c) uall[3 * i + c] = in ? ured[c * nvi + r] : 0.0;
}
void expand_velocity(const Exec& ex, int n, const double* ured, double* uall) {
  size_t tot = (size_t)(2 * n + 1) * (2 * n + 1) * (2 * n + 1);
  ProfScope ps(ex, STOKES_KERNEL_OTHER, 48.0 * tot);
  k_expand<<<cdiv((long long)tot, 256), 256, 0, ex.s>>>(n, ured, uall);  // one thread per node
  SK_CHECK_LAUNCH();
}
__global__ void k_restrict_vel(int n, const double* __restrict__ uall, double* __restrict__ ured) {
  int N = 2 * n + 1, m = 2 * n - 1;
  size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)m * m * m;
  if (r >= tot) return;
  int ix = (int)(r % m) + 1, iy = (int)((r / m) % m) + 1, iz = (int)(r / ((size_t)m * m)) + 1;
  size_t g = (size_t)ix + (size_t)N * (iy + (size_t)N * iz);
  for (int c = 0; c < 3; ++c) ured[c * tot + r] = uall[3 * g + c];
}
void restrict_velocity(const Exec& ex, int n, const double* uall, double* ured) {
  size_t tot = (size_t)(2 * n - 1) * (2 * n - 1) * (2 * n - 1);
  ProfScope ps(ex, STOKES_KERNEL_OTHER, 48.0 * tot);
  k_restrict_vel<<<cdiv((long long)tot, 256), 256, 0, ex.s>>>(n, uall, ured);
  SK_CHECK_LAUNCH();
}

__global__ void k_nonfinite(size_t n, const double* __restrict__ x, int* flag) {
  SK_LOOP(i) {
    if (!isfinite(x[i])) atomicOr(flag, 2);
  }
}
__global__ void k_split_f64(size_t n, const double* __restrict__ x, float* __restrict__ hi,
                            float* __restrict__ lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

void split_f64(const Exec& ex, size_t n, const double* x, float* hi, float* lo) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_BLAS1, 16.0 * n);
  k_split_f64<<<(unsigned)std::min<size_t>(cdiv(n, 256), 1 << 20), 256, 0, ex.s>>>(n, x, hi, lo);
  SK_CHECK_LAUNCH();
}

void count_nonfinite(const Exec& ex, size_t n, const double* x, int* flag) {
  if (!n) return;
  ProfScope ps(ex, STOKES_KERNEL_OTHER, 8.0 * n);
  k_nonfinite<<<SK_GRID(n)>>>(n, x, flag);
  SK_CHECK_LAUNCH();
}

__global__ void k_scalar_sub(double* out, const double* a, const double* b) { *out = *a - *b; }
void scalar_sub(const Exec& ex, double* out, const double* a, const double* b) {
  ProfScope ps(ex, STOKES_KERNEL_OTHER, 24.0);
  k_scalar_sub<<<1, 1, 0, ex.s>>>(out, a, b);
  SK_CHECK_LAUNCH();
}

#define SK_INST1(T)                                                                                     \
  template void dots<T>(const Exec&, const DotScratch&, int, const T* const*, const T* const*, size_t, \
                        double*, int);                                                                       \
  template void axpby<T>(const Exec&, size_t, Coef, const T*, Coef, T*);                               \
  template void cg_update<T>(const Exec&, size_t, Coef, const T*, T*, const T*, T*);                   \
  template void cg_update_rr<T>(const Exec&, const DotScratch&, size_t, Coef, const T*, T*, const T*, T*, double*); \
  template void scale_copy<T>(const Exec&, size_t, Coef, const T*, T*);                                \
  template void lincomb2<T>(const Exec&, size_t, double, const T*, double, const T*, T*);              \
  template void sub_mean<T>(const Exec&, size_t, const double*, double, T*);                           \
  template void sub_ratio<T>(const Exec&, size_t, const double*, const double*, T*);                   \
  template void cheb_first<T>(const Exec&, size_t, int, const T*, const T*, double, T*, T*);             \
  template void cheb_first_il<T>(const Exec&, size_t, int, const T*, const T*, double, T*, T*);          \
  template void to_interleaved<T>(const Exec&, size_t, int, const T*, T*);                              \
  template void to_component_major<T>(const Exec&, size_t, int, const T*, T*);                          \
  template void to_split<T>(const Exec&, size_t, int, const T*, T*, bool, const SplitMap&);             \
  template void from_split<T>(const Exec&, size_t, int, const T*, T*, bool, const SplitMap&);           \
  template void mdot<T>(const Exec&, const DotScratch&, int, const T* const*, const T*, size_t, double*);  \
  template void maxpy<T>(const Exec&, int, const double*, const double*, double, const T* const*, T*, size_t);
SK_INST1(float)
SK_INST1(double)
template void convert<double, float>(const Exec&, size_t, const double*, float*);
template void convert<float, double>(const Exec&, size_t, const float*, double*);
template void convert<double, double>(const Exec&, size_t, const double*, double*);
template void add_convert<float, double>(const Exec&, size_t, const float*, double*);
template void add_convert<double, double>(const Exec&, size_t, const double*, double*);

}  // namespace sk
