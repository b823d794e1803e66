// Allocation-free application of the augmented velocity operator
//   y = A x + gamma mu B^T M_Q^{-1} B x
// for callers that must not allocate device memory once they are running
// (a host loop that owns a fixed device-memory budget, or code that runs while
// another framework owns the device allocator). The paper has no counterpart;
// the arithmetic is exactly that of stokes_apply(ctx, STOKES_OP_AGAMMA, ...).
//
// The four work vectors live in one file-scope __device__ array of fixed
// size. Every device that loads this library holds that array until the
// process exits, every call shares it, and a call leaves its contents behind;
// all four vectors are fully overwritten before they are read, so nothing
// needs clearing. Calls whose kernels overlap on the GPU (for example two
// streams, or two contexts used from two threads at once) race on the array.
#include <cmath>
#include <exception>
#include <mutex>
#include <new>
#include <string>

#include "internal.h"

namespace {

constexpr size_t kNoAllocMaxP1 = (size_t)1 << 20;  // pressure nodes per call (n <= 100)
constexpr int kNoAllocVectors = 4;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocVectors * kNoAllocMaxP1];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
// In host code g_noalloc_scratch only names a host-side shadow symbol; its
// device address has to come from the runtime.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" stokes_status stokes_apply_agamma_noalloc(stokes_ctx* c, const double* x, double* y) {
  using namespace sk;
  set_last_error("");
  if (!c || !x || !y) {
    set_last_error("stokes_apply_agamma_noalloc: null argument");
    return STOKES_ERR_ARG;
  }
  const size_t np = (size_t)c->lv[0].np;
  if (np > kNoAllocMaxP1) {
    set_last_error("stokes_apply_agamma_noalloc: " + std::to_string(np) +
                   " pressure nodes exceed the fixed work array (at most " + std::to_string(kNoAllocMaxP1) +
                   ", i.e. n <= 100)");
    return STOKES_ERR_ARG;
  }
  double* base = nullptr;
  cudaError_t ae = scratch_address(&base);
  if (ae != cudaSuccess) {
    set_last_error(std::string("stokes_apply_agamma_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(ae));
    return STOKES_ERR_CUDA;
  }
  try {
    Exec ex{c->ex.s, nullptr};  // no profiling events: nothing is created per call
    bsr3_apply<double>(ex, c->A, x, y, (const double*)nullptr);
    if (c->gamma > 0.0) {
      double* bx = base;
      double* mb = base + kNoAllocMaxP1;
      double* d = base + 2 * kNoAllocMaxP1;
      double* xt = base + 3 * kNoAllocMaxP1;
      b_apply<double>(ex, c->B, x, bx, (const double*)nullptr, 1.0);
      // M_Q^{-1} bx: Chebyshev-Jacobi on sigma(D^{-1} M_Q) in [1/2, 5/2], from zero,
      // the same steps and coefficients as the allocating path
      const double lo = 0.5, hi = 2.5;
      const int steps = c->opt.mass_steps_al > 1 ? c->opt.mass_steps_al : 1;
      double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta, rho = 1.0 / sigma;
      double* xa = mb;
      double* xb = xt;
      cheb_first<double>(ex, np, 1, c->MQ_dinv64, bx, 1.0 / theta, d, xa);
      for (int k = 1; k < steps; ++k) {
        double rn = 1.0 / (2.0 * sigma - rho);
        spmv_cheb<double>(ex, c->MQ, 1, bx, xa, d, xb, c->MQ_dinv64, rn * rho, 2.0 * rn / delta,
                          STOKES_KERNEL_SPMV_P1);
        double* t = xa;
        xa = xb;
        xb = t;
        rho = rn;
      }
      bt_apply<double>(ex, c->Bt, xa, y, (const double*)nullptr, y, c->gamma * c->mu);
    }
    cudaError_t se = cudaStreamSynchronize(c->ex.s);
    if (se != cudaSuccess) {
      set_last_error(std::string("stokes_apply_agamma_noalloc: ") + cudaGetErrorString(se));
      return STOKES_ERR_CUDA;
    }
  } catch (const sk::Error& e) {
    set_last_error(e.what());
    return (stokes_status)e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("stokes_apply_agamma_noalloc: host allocation failed");
    return STOKES_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(std::string("stokes_apply_agamma_noalloc: ") + e.what());
    return STOKES_ERR_CUDA;
  } catch (...) {
    set_last_error("stokes_apply_agamma_noalloc: unknown exception");
    return STOKES_ERR_CUDA;
  }
  return STOKES_OK;
}
