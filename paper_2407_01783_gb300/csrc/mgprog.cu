// The coarse levels of a V-cycle in one cooperative kernel.
//
// Below the finest level the V-cycle's products are small (10^5 rows and
// fewer), so launching each smoothing step, residual, transfer and the coarse
// solve as its own kernel costs more in launch latency than in memory
// traffic. Here the whole sequence (an MgProgram of steps built once per
// context, V-cycle kind and precision, with fixed buffers) runs inside one
// cooperative launch: every block walks the steps in order, each step spreads
// its rows over the whole grid, and a grid-wide barrier separates dependent
// steps. The barrier is a counter in device memory; a block that waits longer
// than kMgSpinLimit polls sets the context's error flag (STOKES_ERR_TIMEOUT
// on the host) and leaves the kernel instead of waiting forever.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace sk {

constexpr int kMgBlock = 512;
constexpr int kMgG = 4;                       // threads per CSR row
constexpr long long kMgSpinLimit = 1LL << 23; // polls (spinning, then ~128 ns sleeps) before giving up

struct MgOpDev {
  int kind, nr, rows, m;
  const int* rp;
  const int* col;
  const void* val;
  const void* b;
  const void* xin;
  void* d;
  void* y;
  const void* dinv;
  double c1, c2;
};
static_assert(sizeof(MgOpDev) % 8 == 0, "MgOpDev layout");

// Grid barrier on a monotone counter: barrier k completes when the counter
// reaches k * gridDim.x. Returns false if this block gave up waiting.
__device__ __forceinline__ bool mg_grid_sync(unsigned* bar, unsigned target, int* flag) {
  __shared__ int ok_;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok_ = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    long long polls = 0;
    while (true) {
      const unsigned v = *(volatile unsigned*)bar;
      if (v >= target) break;
      if (flag && (*(volatile int*)flag & 4)) {  // another block already gave up
        ok_ = 0;
        break;
      }
      if (++polls > kMgSpinLimit) {
        if (flag) atomicOr(flag, 4);
        ok_ = 0;
        break;
      }
      if (polls > 4096) __nanosleep(128);  // spin first: most barriers complete within a microsecond
    }
    __threadfence();
  }
  __syncthreads();
  return ok_ != 0;
}

template <class T, int NR>
__device__ __forceinline__ void mg_csr(const MgOpDev& o) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  constexpr int RW = 32 / kMgG;  // rows per warp and iteration
  const int sub = lane % kMgG;
  const T* __restrict__ val = (const T*)o.val;
  const T* __restrict__ x = (const T*)o.xin;
  const size_t xs = (size_t)o.m;  // column-space length (component stride of x)
  const size_t ys = (size_t)o.rows;
  for (int r0 = gw * RW; r0 < o.rows; r0 += nw * RW) {
    const int row = r0 + lane / kMgG;
    const bool valid = row < o.rows;
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = T(0);
    if (valid) {
      const int e = o.rp[row + 1];
      for (int k = o.rp[row] + sub; k < e; k += kMgG) {
        const int cidx = o.col[k];
        const T a = val[k];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] += a * __ldcg(&x[r * xs + cidx]);  // written by earlier steps
      }
    }
#pragma unroll
    for (int off = kMgG / 2; off > 0; off >>= 1)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
    if (!valid || sub != 0) continue;
    T* y = (T*)o.y;
    switch (o.kind) {
      case 1:  // y = A x
#pragma unroll
        for (int r = 0; r < NR; ++r) y[r * ys + row] = acc[r];
        break;
      case 2:  // y += A x
#pragma unroll
        for (int r = 0; r < NR; ++r) y[r * ys + row] = __ldcg(&y[r * ys + row]) + acc[r];
        break;
      case 3: {  // y = b - A x
        const T* b = (const T*)o.b;
#pragma unroll
        for (int r = 0; r < NR; ++r) y[r * ys + row] = __ldcg(&b[r * ys + row]) - acc[r];
        break;
      }
      default: {  // Chebyshev step: d = c1 d + c2 D^-1 (b - A x_in), y = x_in + d
        const T* b = (const T*)o.b;
        T* d = (T*)o.d;
        const T di = ((const T*)o.dinv)[row];
        const T c1 = (T)o.c1, c2 = (T)o.c2;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const size_t i = r * ys + row;
          const T dn = c1 * __ldcg(&d[i]) + c2 * di * (__ldcg(&b[i]) - acc[r]);
          d[i] = dn;
          y[i] = __ldcg(&x[i]) + dn;
        }
        break;
      }
    }
  }
}

// y = M b for the dense coarsest-level inverse (one warp per row)
template <class T, int NR>
__device__ __forceinline__ void mg_dense(const MgOpDev& o) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const T* __restrict__ M = (const T*)o.val;
  const T* __restrict__ b = (const T*)o.b;
  T* y = (T*)o.y;
  const int m = o.m;
  for (int row = gw; row < m; row += nw) {
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = T(0);
    for (int j = lane; j < m; j += 32) {
      const T a = M[(size_t)row * m + j];
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r] += a * __ldcg(&b[(size_t)r * m + j]);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < NR; ++r) y[(size_t)r * m + row] = acc[r];
  }
}

// first Chebyshev step from zero: d = y = c D^-1 b (per component)
template <class T>
__device__ __forceinline__ void mg_cheb_first(const MgOpDev& o) {
  const T* b = (const T*)o.b;
  const T* dinv = (const T*)o.dinv;
  T* d = (T*)o.d;
  T* y = (T*)o.y;
  const T c = (T)o.c1;
  const size_t len = (size_t)o.rows * o.nr;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
    const T v = c * dinv[i % o.rows] * __ldcg(&b[i]);
    d[i] = v;
    y[i] = v;
  }
}

template <class T>
__global__ void __launch_bounds__(kMgBlock) k_mg_program(const MgOpDev* __restrict__ ops, int nops, unsigned* bar,
                                                        int* flag) {
  for (int k = 0; k < nops; ++k) {
    const MgOpDev o = ops[k];
    switch (o.kind) {
      case 0: mg_cheb_first<T>(o); break;
      case 5:
        if (o.nr == 3) mg_dense<T, 3>(o);
        else mg_dense<T, 1>(o);
        break;
      default:
        if (o.nr == 3) mg_csr<T, 3>(o);
        else mg_csr<T, 1>(o);
        break;
    }
    if (k + 1 < nops && !mg_grid_sync(bar, (unsigned)(k + 1) * gridDim.x, flag)) return;
  }
}

// A barrier that can never complete (its target counts one block more than
// the grid has): every block's wait runs out after kMgSpinLimit polls, sets the
// timeout bit and returns. Used by stokes_check_bounded_wait.
__global__ void k_unreachable_barrier(unsigned* bar, int* flag) {
  (void)mg_grid_sync(bar, gridDim.x + 1, flag);
}

void bounded_wait_check(const Exec& ex, unsigned* bar) {
  SK_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), ex.s));
  k_unreachable_barrier<<<2, 32, 0, ex.s>>>(bar, ex.flag);
  SK_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void MgProgram::add(const MgOp& op) {
  SK_REQUIRE(op.nr == 1 || op.nr == 3, STOKES_ERR_ARG, "multigrid program: 1 or 3 components");
  ops.push_back(op);
}

void MgProgram::finalize(Arena& ar, bool f32) {
  this->f32 = f32;
  std::vector<MgOpDev> h(ops.size());
  int max_rows = 1;
  for (size_t k = 0; k < ops.size(); ++k) {
    const MgOp& o = ops[k];
    MgOpDev& d = h[k];
    std::memset(&d, 0, sizeof(d));
    d.kind = o.kind;
    d.nr = o.nr;
    d.rows = o.rows;
    d.m = o.m;
    d.rp = o.rp;
    d.col = o.col;
    d.val = o.val;
    d.b = o.b;
    d.xin = o.xin;
    d.d = o.d;
    d.y = o.y;
    d.dinv = o.dinv;
    d.c1 = o.c1;
    d.c2 = o.c2;
    max_rows = std::max(max_rows, o.kind == 5 ? o.m * 32 / kMgG : o.rows);
  }
  dev_ops = ar.alloc<MgOpDev>(h.size());
  SK_CUDA(cudaMemcpy(dev_ops, h.data(), sizeof(MgOpDev) * h.size(), cudaMemcpyHostToDevice));
  bar = ar.alloc<unsigned>(1);
  int dev = 0, sms = 0, occ = 0, coop = 0;
  SK_CUDA(cudaGetDevice(&dev));
  SK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SK_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  SK_REQUIRE(coop, STOKES_ERR_CUDA, "device does not support cooperative launches");
  if (f32)
    SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mg_program<float>, kMgBlock, 0));
  else
    SK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mg_program<double>, kMgBlock, 0));
  SK_REQUIRE(occ >= 1, STOKES_ERR_CUDA, "multigrid program kernel cannot be resident");
  // enough blocks for the largest step, at most one per SM: every barrier
  // costs one atomic per block, so fewer, larger blocks keep it short
  const int want = cdiv((long long)max_rows * kMgG, kMgBlock);
  grid = std::max(1, std::min(want, sms));
}

void MgProgram::launch(const Exec& ex) const {
  SK_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), ex.s));
  int nops = (int)ops.size();
  MgOpDev* p = dev_ops;
  unsigned* b = bar;
  int* fl = ex.flag;
  void* args[] = {&p, &nops, &b, &fl};
  ProfScope ps(ex, STOKES_KERNEL_COARSE_CYCLE, bytes);
  if (f32)
    SK_CUDA(cudaLaunchCooperativeKernel((const void*)k_mg_program<float>, grid, kMgBlock, args, 0, ex.s));
  else
    SK_CUDA(cudaLaunchCooperativeKernel((const void*)k_mg_program<double>, grid, kMgBlock, args, 0, ex.s));
}

}  // namespace sk
