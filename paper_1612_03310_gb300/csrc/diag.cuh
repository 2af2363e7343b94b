// diag.cuh -- diagnostics of a running simulation: bunch sampling and the
// bunching factor (input group "bunch-sampling"; bunching factor
// |<exp(i k_b z)>|), and the frequency-resolved radiated power (FEL-OUTPUT
// radiation-power with wavelengths).  Every sum is FP64 and runs in a fixed
// order (per-block partials, then one ordered pass), so repeated calls give
// identical results.
#pragma once
#include "common.cuh"
#include "field_kernels.cuh"

namespace mithra {

constexpr int kBunchSums = 15;  // x, y, z, ux, uy, uz; their squares; cos, sin; count

// Block-wide sum of one double per thread (blockDim 256); every thread gets it.
__device__ inline double block_sum256(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < 8; ++w) s += red[w];
  return s;
}

// A recording sample is due after the step whose device counter n has
// (n - first) % every == every - 1.
__device__ inline bool bunch_due(const StepState* __restrict__ st, long long first, int every) {
  return every <= 0 || (st->n - first) % every == every - 1;
}

// Pass 1: per-block sums over the particles not lost, positions in FP64 from
// (cell, fraction).  With st, only when a recording sample is due.

template <typename T, typename U>
__global__ void __launch_bounds__(256) k_bunch_partial(PicP<T> p, Parts<T, U> P, long long np,
                                                       double kb, double* __restrict__ part,
                                                       const StepState* __restrict__ st = nullptr,
                                                       long long first = 0, int every = 0) {
  if (st && !bunch_due(st, first, every)) return;
  __shared__ double red[8];
  double acc[kBunchSums];
  for (int m = 0; m < kBunchSums; ++m) acc[m] = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < np;
       q += (long long)gridDim.x * blockDim.x) {
    const int cell = P.cell[q];
    if (cell < 0) continue;
    int i, j, k;
    decode_cell(p, cell, &i, &j, &k);
    const double v[6] = {p.x0 + ((double)i + (double)P.fx[q]) * p.dxd,
                         p.y0 + ((double)j + (double)P.fy[q]) * p.dyd,
                         p.z0 + ((double)k + (double)P.fz[q]) * p.dzd,
                         u_dbl(P.ux[q]), u_dbl(P.uy[q]), u_dbl(P.uz[q])};
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      acc[a] += v[a];
      acc[6 + a] += v[a] * v[a];
    }
    double sn, cs;
    sincos(kb * v[2], &sn, &cs);
    acc[12] += cs;
    acc[13] += sn;
    acc[14] += 1.0;
  }
  for (int m = 0; m < kBunchSums; ++m) {
    const double s = block_sum256(acc[m], red);
    if (threadIdx.x == 0) part[blockIdx.x * kBunchSums + m] = s;
  }
}

// Pass 2: the block sums in block order, then means, rms spreads and the
// bunching factor into out[14] (layout of mithra_bunch_stats).
// With st: the sample goes to record (n - first) / every of out (15 values:
// the step count after the sampled step, then the 14 statistics) when due
// and within cap records.
__global__ void k_bunch_final(const double* __restrict__ part, int nblocks,
                              double* __restrict__ out,
                              const StepState* __restrict__ st = nullptr, long long first = 0,
                              int every = 0, long long cap = 0) {
  if (st) {
    if (!bunch_due(st, first, every)) return;
    const long long r = (st->n - first) / every;
    if (r >= cap) return;
    if (threadIdx.x == 0) out[r * 15] = (double)(st->n + 1);
    out += r * 15 + 1;
  }
  __shared__ double tot[kBunchSums];
  const int m = threadIdx.x;
  if (m < kBunchSums) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[b * kBunchSums + m];
    tot[m] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double n = tot[14];
    for (int a = 0; a < 6; ++a) {
      const double mean = n > 0 ? tot[a] / n : 0.0;
      const double var = n > 0 ? tot[6 + a] / n - mean * mean : 0.0;
      out[a] = mean;
      out[6 + a] = var > 0 ? sqrt(var) : 0.0;
    }
    out[12] = n > 0 ? sqrt(tot[12] * tot[12] + tot[13] * tot[13]) / n : 0.0;
    out[13] = n;
  }
}

// Running Fourier sums of the lab fields at plane kp (interior vertices v =
// (j-1)(nx-2) + (i-1)), one step: the lab time of the sample is
// t' = gamma0 (t + beta0 z_p / c) with t = t0 + (n + 1/2) dt from the device
// clock, and for each observed angular frequency omega[m]
//   acc[((m nv) + v) 8 + 2f + {0,1}] += F_f (cos, -sin)(omega[m] t') dt',
// F = (E'_x, E'_y, B'_x, B'_y) the lab transformation of k_power.
constexpr int kMaxSpectrum = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_spectrum_accumulate(
    PicP<T> p, const V4<T>* __restrict__ pn, const V4<T>* __restrict__ D, int kp, double g0,
    double b0, double zp, const StepState* __restrict__ st, int nf,
    const double* __restrict__ omega, double* __restrict__ acc,
    long long* __restrict__ samples) {
  __shared__ double2 ph[kMaxSpectrum];
  const double t = p.t0 + ((double)st->n + 0.5) * p.dt;
  const double tl = g0 * (t + b0 * zp / kC);
  const double dtl = g0 * p.dt;
  const double b0c = b0 / kC;
  for (int m = threadIdx.x; m < nf; m += blockDim.x) {
    double sn, cs;
    sincos(omega[m] * tl, &sn, &cs);
    ph[m] = make_double2(cs * dtl, -sn * dtl);
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) *samples += 1;
  const int nvx = p.nx - 2;
  const long long nv = (long long)nvx * (p.ny - 2);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv;
       v += (long long)gridDim.x * blockDim.x) {
    const int i = 1 + (int)(v % nvx), j = 1 + (int)(v / nvx);
    T E[3], B[3];
    eb_vertex(p, pn, D, cidx(i, j, kp, p.nx, p.nxy), E, B);
    const double Ex = E[0], Ey = E[1], Bx = B[0], By = B[1];
    const double F[4] = {g0 * (Ex + b0 * kC * By), g0 * (Ey - b0 * kC * Bx),
                         g0 * (Bx - b0c * Ey), g0 * (By + b0c * Ex)};
    for (int m = 0; m < nf; ++m) {
      double* a = acc + ((long long)m * nv + v) * 8;
      const double2 e = ph[m];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        a[2 * f] += F[f] * e.x;
        a[2 * f + 1] += F[f] * e.y;
      }
    }
  }
}

// Energy through the plane per unit observed angular frequency, one block per
// frequency, vertices summed in a fixed order:
//   out[m] = (1/pi) sum_v Re(E~x B~y* - E~y B~x*) dx dy / mu0.
__global__ void __launch_bounds__(256) k_spectrum_density(const double* __restrict__ acc,
                                                          long long nv, double scale,
                                                          double* __restrict__ out) {
  __shared__ double red[8];
  const int m = blockIdx.x;
  double s = 0.0;
  for (long long v = threadIdx.x; v < nv; v += blockDim.x) {
    const double* a = acc + ((long long)m * nv + v) * 8;
    s += (a[0] * a[6] + a[1] * a[7]) - (a[2] * a[4] + a[3] * a[5]);
  }
  const double tot = block_sum256(s, red);
  if (threadIdx.x == 0) out[m] = tot * scale;
}

}  // namespace mithra
