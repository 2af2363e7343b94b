// noalloc.cu -- radiated power through one vertex plane from caller-owned
// device arrays, without allocating any device or pinned memory.
//
// Some callers cannot call cudaMalloc: a custom operator inside another
// framework whose caching allocator owns all device memory (a second
// allocator beside it fragments the device and can fail once that allocator
// has reserved the rest), or a real-time loop that must not stall on the
// driver's allocator.  For them this file keeps its scratch memory in one
// file-scope device array of fixed size instead of allocating it.
//
// Scratch: kRows + 1 doubles (64 KiB).  Slots 0 .. ny-1 take one partial sum
// per grid row j (rows 1 .. ny-2 are used), slot kRows the total.  Every call
// writes every slot it later reads, so nothing has to start at zero; the
// array keeps the last call's values.  The array is shared by all calls on a
// device: two calls whose work overlaps on the GPU (different streams, no
// ordering between them) race on it and must be serialised by the caller.
//
// The call waits for its own work (it synchronises the stream it is given)
// and copies the result to the caller's host variable before it returns.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "mithra.h"
#include "common.cuh"
#include "field_kernels.cuh"

using namespace mithra;

namespace mithra {
void set_thread_error(const std::string& msg);  // mithra_last_error(NULL)
}

namespace {

constexpr int kRows = 8192;  // largest ny accepted is kRows

static __device__ __align__(256) double g_scratch[kRows + 1];

mithra_status na_fail(mithra_status st, const std::string& msg) {
  mithra::set_thread_error(msg);
  return st;
}

// Device address of g_scratch in the current context, looked up on every
// call with the caller's device current (the host-side name g_scratch is only
// a stand-in for the symbol, not a device address).  cudaGetSymbolAddress
// allocates nothing; looking it up each time keeps the address right after a
// cudaDeviceReset or in a context other than the device's primary one, where
// the module is loaded again at another address.  The first call in a
// context may load the module.
mithra_status scratch_of_current_context(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess)
    return na_fail(MITHRA_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = static_cast<double*>(p);
  return MITHRA_OK;
}

// Pass 1: one block per interior row j, the lab-frame Poynting flux summed
// over interior i (same transformation as k_power), written to rows[j].
template <typename T>
__global__ void __launch_bounds__(256) k_plane_rows(PicP<T> p, const V4<T>* __restrict__ pn,
                                                    const V4<T>* __restrict__ D, int kp,
                                                    double g0, double b0,
                                                    double* __restrict__ rows) {
  const int j = 1 + blockIdx.x;
  const double b0c = b0 / kC;
  double part = 0.0;
  for (int i = 1 + threadIdx.x; i <= p.nx - 2; i += blockDim.x) {
    T E[3], B[3];
    eb_vertex(p, pn, D, cidx(i, j, kp, p.nx, p.nxy), E, B);
    const double Ex = E[0], Ey = E[1], Bx = B[0], By = B[1];
    const double exl = g0 * (Ex + b0 * kC * By);
    const double eyl = g0 * (Ey - b0 * kC * Bx);
    const double bxl = g0 * (Bx - b0c * Ey);
    const double byl = g0 * (By + b0c * Ex);
    part += exl * byl - eyl * bxl;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    rows[j] = v;
  }
}

// Pass 2: one block adds rows 1 .. ny-2 in a fixed order into slot kRows.
__global__ void __launch_bounds__(256) k_plane_total(const double* __restrict__ rows, int ny,
                                                     double scale, double* __restrict__ total) {
  double part = 0.0;
  for (int j = 1 + threadIdx.x; j <= ny - 2; j += blockDim.x) part += rows[j];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    *total = v * scale;
  }
}

template <typename T>
PicP<T> plane_params(const mithra_grid* g, const LoV4* lo) {
  PicP<T> p{};
  p.plo = lo;
  p.nx = g->nx; p.ny = g->ny; p.nz = g->nz;
  p.nxy = (long long)g->nx * g->ny;
  p.inv2dx = (T)(0.5 / g->dx); p.inv2dy = (T)(0.5 / g->dy); p.inv2dz = (T)(0.5 / g->dz);
  p.invdt = (T)(1.0 / g->dt);
  p.dxd = g->dx; p.dyd = g->dy;
  return p;
}

template <typename T>
mithra_status run(const mithra_grid* g, double gamma0, const void* psi, const void* lo,
                  const void* incr, int kp, double* p_lab, cudaStream_t stream,
                  double* scratch) {
  const double b0 = std::sqrt(1.0 - 1.0 / (gamma0 * gamma0));
  const PicP<T> p = plane_params<T>(g, static_cast<const LoV4*>(lo));
  k_plane_rows<T><<<g->ny - 2, 256, 0, stream>>>(p, static_cast<const V4<T>*>(psi),
                                                static_cast<const V4<T>*>(incr), kp, gamma0, b0,
                                                scratch);
  k_plane_total<<<1, 256, 0, stream>>>(scratch, g->ny, g->dx * g->dy / kMu0, scratch + kRows);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(MITHRA_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(p_lab, scratch + kRows, sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return na_fail(MITHRA_ECUDA, std::string("copy-out: ") + cudaGetErrorString(e));
  if (!std::isfinite(*p_lab)) return na_fail(MITHRA_ENUMERIC, "NaN or Inf in the power sum");
  return MITHRA_OK;
}

}  // namespace

extern "C" {

mithra_status mithra_plane_power_noalloc(const mithra_grid* grid, double gamma0,
                                         mithra_precision precision, const void* psi_newest,
                                         const void* lo_newest, const void* increment,
                                         int32_t k_plane, double* p_lab, void* cuda_stream) {
  if (!grid || !psi_newest || !increment || !p_lab)
    return na_fail(MITHRA_EINVAL, "grid, arrays and p_lab must not be NULL");
  if (grid->nx < 4 || grid->ny < 4 || grid->nz < 4 || !(grid->dx > 0) || !(grid->dy > 0) ||
      !(grid->dz > 0) || !(grid->dt > 0))
    return na_fail(MITHRA_EINVAL, "bad grid");
  if (grid->ny > kRows)
    return na_fail(MITHRA_EINVAL, "ny exceeds the fixed scratch of 8192 rows of this entry point");
  if ((int64_t)grid->nx * grid->ny * grid->nz >= (int64_t)1 << 31)
    return na_fail(MITHRA_EINVAL, "grid has >= 2^31 vertices");
  if (k_plane < 1 || k_plane > grid->nz - 2) return na_fail(MITHRA_EINVAL, "k_plane outside [1, nz-2]");
  if (!(gamma0 > 1.0)) return na_fail(MITHRA_EINVAL, "gamma0 must be > 1");
  if (precision != MITHRA_P64 && precision != MITHRA_P32 && precision != MITHRA_P32_U64 &&
      precision != MITHRA_P32_C)
    return na_fail(MITHRA_EINVAL, "bad precision");
  if (lo_newest && (precision == MITHRA_P64 || precision == MITHRA_P32))
    return na_fail(MITHRA_EINVAL, "lo_newest is only for the compensated forms P32_C, P32_U64");
  double* scratch = nullptr;
  mithra_status st = scratch_of_current_context(&scratch);
  if (st != MITHRA_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  if (precision == MITHRA_P64)
    return run<double>(grid, gamma0, psi_newest, nullptr, increment, k_plane, p_lab, stream,
                       scratch);
  return run<float>(grid, gamma0, psi_newest, lo_newest, increment, k_plane, p_lab, stream,
                    scratch);
}

}  // extern "C"
