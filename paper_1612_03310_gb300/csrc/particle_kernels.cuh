// particle_kernels.cuh -- macroparticles: set-up, gather + undulator + Boris
// push (Eq. BorisScheme, Eq. fieldInterpolation, Sec. "Undulator Field"),
// current and charge deposition (Sec. "Current Deposition",
// Eq. currentIntegral), and the binning of particles into cell tiles.
#pragma once
#include "common.cuh"
#include "field_kernels.cuh"

namespace mithra {

// --- math in the particle's precision ------------------------------------
__device__ inline void sincos_t(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ inline void sincos_t(double a, double* s, double* c) { sincos(a, s, c); }
__device__ inline float cosh_t(float a) { return coshf(a); }
__device__ inline double cosh_t(double a) { return cosh(a); }
__device__ inline float sinh_t(float a) { return sinhf(a); }
__device__ inline double sinh_t(double a) { return sinh(a); }
__device__ inline float exp_t(float a) { return expf(a); }
__device__ inline double exp_t(double a) { return exp(a); }

// Rest-frame undulator field at (y, z_abs, t).  The lab distance past the
// entrance, zeta = gamma0 (z + beta0 c t) - z'_ent, and its reduction modulo
// lambda_u are FP64; the trigonometric and hyperbolic factors are in T.
template <typename T>
__device__ inline void undulator_field(const PicP<T>& p, T y, double zabs, double t, T E[3],
                                       T B[3]) {
  E[0] = E[1] = E[2] = (T)0;
  B[0] = B[1] = B[2] = (T)0;
  if (!p.und_on) return;
  const double zeta = p.g0 * (zabs + p.b0c * t) - p.zent;
  const T ky = p.ku * y;
  const T ch = cosh_t(ky), sh = sinh_t(ky);
  T by, bz;
  const bool before = zeta < 0.0;
  const bool after = p.L > 0.0 && zeta > p.L;
  if (before || after) {
    if (!p.fringe) return;
    const T a = (T)(p.ku_d * (before ? zeta : zeta - p.L));
    const T e = exp_t((T)(-0.5) * a * a);
    by = p.B0 * ch * a * e;
    bz = p.B0 * sh * e;
  } else {
    const double zr = zeta - p.lam_u * rint(zeta * p.inv_lam_u);
    T s, c;
    sincos_t((T)(p.ku_d * zr), &s, &c);
    by = p.B0 * ch * s;
    bz = p.B0 * sh * c;
  }
  E[0] = p.ex_fac * by;
  B[1] = p.by_fac * by;
  B[2] = bz;
}

// Trilinear gather of E, B (Eq. fieldInterpolation, w0 = 1 - f, w1 = f) at a
// particle in cell (i, j, k) with fractions f, evaluating E, B at the eight
// vertices from the potentials.
template <typename T>
__device__ inline void gather_eb(const PicP<T>& p, const V4<T>* __restrict__ pn,
                                 const V4<T>* __restrict__ D, int i, int j, int k, T fx, T fy,
                                 T fz, T E[3], T B[3]) {
  E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = (T)0;
  const T wx[2] = {(T)1 - fx, fx}, wy[2] = {(T)1 - fy, fy}, wz[2] = {(T)1 - fz, fz};
#pragma unroll
  for (int K = 0; K < 2; ++K)
#pragma unroll
    for (int J = 0; J < 2; ++J)
#pragma unroll
      for (int I = 0; I < 2; ++I) {
        T e[3], b[3];
        eb_vertex(p, pn, D, cidx(i + I, j + J, k + K, p.nx, p.nxy), e, b);
        const T w = wx[I] * wy[J] * wz[K];
        E[0] += w * e[0]; E[1] += w * e[1]; E[2] += w * e[2];
        B[0] += w * b[0]; B[1] += w * b[1]; B[2] += w * b[2];
      }
}

// Boris rotation and kicks (Eq. BorisScheme) for charge-to-mass qm folded
// into h = qm dtb / (2c) and an = qm dtb / 2, in the momentum type U; gamma
// of t1 in FP64.
template <typename T, typename U>
__device__ inline void boris(const PicP<T>& p, U u[3], const T Ef[3], const T Bf[3]) {
  const U h = (U)p.h;
  const U E[3] = {(U)Ef[0], (U)Ef[1], (U)Ef[2]};
  const U B[3] = {(U)Bf[0], (U)Bf[1], (U)Bf[2]};
  const U t1x = u[0] + h * E[0], t1y = u[1] + h * E[1], t1z = u[2] + h * E[2];
  const double g1 = sqrt(1.0 + (double)t1x * t1x + (double)t1y * t1y + (double)t1z * t1z);
  const U al = (U)(p.an / g1);
  const U t2x = t1x + al * (t1y * B[2] - t1z * B[1]);
  const U t2y = t1y + al * (t1z * B[0] - t1x * B[2]);
  const U t2z = t1z + al * (t1x * B[1] - t1y * B[0]);
  const U f = (U)2 * al / ((U)1 + al * al * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
  const U sx = f * B[0], sy = f * B[1], sz = f * B[2];
  const U t3x = t1x + (t2y * sz - t2z * sy);
  const U t3y = t1y + (t2z * sx - t2x * sz);
  const U t3z = t1z + (t2x * sy - t2y * sx);
  u[0] = t3x + h * E[0];
  u[1] = t3y + h * E[1];
  u[2] = t3z + h * E[2];
}

__device__ inline bool valid_cell(int i, int j, int k, int nx, int ny, int nz) {
  return i >= 1 && i <= nx - 3 && j >= 1 && j <= ny - 3 && k >= 1 && k <= nz - 3;
}

template <typename T>
__device__ inline int tile_key(const PicP<T>& p, int i, int j, int k) {
  return ((k / kTile) * p.nty + (j / kTile)) * p.ntx + (i / kTile);
}

// Rank of this lane's key among the keys already counted: lanes of a warp
// with equal keys share one atomic (warp-level binning).
__device__ inline int bin_rank(int* __restrict__ count, int key) {
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count + key, __popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

template <typename T>
__device__ inline void dep_add(V4<T>* a, T x, T y, T z, T w);
template <>
__device__ inline void dep_add<float>(V4<float>* a, float x, float y, float z, float w) {
  atomicAdd(reinterpret_cast<float4*>(a), make_float4(x, y, z, w));
}
template <>
__device__ inline void dep_add<double>(V4<double>* a, double x, double y, double z, double w) {
  if (x != 0.0) atomicAdd(&a->x, x);
  if (y != 0.0) atomicAdd(&a->y, y);
  if (z != 0.0) atomicAdd(&a->z, z);
  if (w != 0.0) atomicAdd(&a->w, w);
}

template <typename T>
__device__ inline void deposit_cic(const PicP<T>& p, V4<T>* __restrict__ src, int i, int j,
                                   int k, T fx, T fy, T fz, T jx, T jy, T jz, T rho) {
  const T wx[2] = {(T)1 - fx, fx}, wy[2] = {(T)1 - fy, fy}, wz[2] = {(T)1 - fz, fz};
#pragma unroll
  for (int K = 0; K < 2; ++K)
#pragma unroll
    for (int J = 0; J < 2; ++J)
#pragma unroll
      for (int I = 0; I < 2; ++I) {
        const T w = wx[I] * wy[J] * wz[K];
        dep_add(src + cidx(i + I, j + J, k + K, p.nx, p.nxy), w * jx, w * jy, w * jz, w * rho);
      }
}

// Splits an FP64 offset (in cells, relative to cell index c0) into the cell
// index and the fraction in [0, 1).
__device__ inline int split_cell(int c0, double s, double* frac) {
  const double fl = floor(s);
  *frac = s - fl;
  return c0 + (int)fl;
}

// One field step of every particle: n_sub Boris steps with the grid E, B at
// t = (n+1/2) dt held fixed and the undulator at each sub-step time, then the
// deposit of J^{n+1} at the mid point of the path and rho^{n+3/2} at the end,
// and the key/rank of the particle's new tile for the re-sort.
template <typename T, typename U>
__global__ void __launch_bounds__(256) k_push(PicP<T> p, const StepState* __restrict__ st,
                                              const V4<T>* __restrict__ pn,
                                              const V4<T>* __restrict__ D,
                                              V4<T>* __restrict__ src, Parts<T, U> P, long long np,
                                              int* __restrict__ count, int* __restrict__ key,
                                              int* __restrict__ rank,
                                              long long* __restrict__ lost_ctr) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  int cell = P.cell[q];
  int kk = p.nkeys;  // bucket of lost particles
  if (cell >= 0) {
    int i = cell % p.nx, j = (cell / p.nx) % p.ny, k = cell / (int)p.nxy;
    T f[3] = {P.fx[q], P.fy[q], P.fz[q]};
    U u[3] = {P.ux[q], P.uy[q], P.uz[q]};
    const int i0 = i, j0 = j, k0 = k;
    const T f0x = f[0], f0y = f[1], f0z = f[2];
    double disp[3] = {0.0, 0.0, 0.0};  // displacement in cells
    const double th = p.t0 + ((double)st->n + 0.5) * p.dt;
    bool ok = true;
    for (int m = 0; m < p.n_sub && ok; ++m) {
      T E[3], B[3], Eu[3], Bu[3];
      gather_eb(p, pn, D, i, j, k, f[0], f[1], f[2], E, B);
      const double zabs = p.z0 + ((double)k + (double)f[2]) * p.dzd;
      const T y = (T)(p.y0 + ((double)j + (double)f[1]) * p.dyd);
      undulator_field(p, y, zabs, th + m * p.dtb, Eu, Bu);
      for (int a = 0; a < 3; ++a) { E[a] += Eu[a]; B[a] += Bu[a]; }
      boris(p, u, E, B);
      const double g = sqrt(1.0 + (double)u[0] * u[0] + (double)u[1] * u[1] + (double)u[2] * u[2]);
      const double d[3] = {p.cdtb_dx * u[0] / g, p.cdtb_dy * u[1] / g, p.cdtb_dz * u[2] / g};
      double fr[3];
      i = split_cell(i, (double)f[0] + d[0], &fr[0]);
      j = split_cell(j, (double)f[1] + d[1], &fr[1]);
      k = split_cell(k, (double)f[2] + d[2], &fr[2]);
      f[0] = to_frac<T>(fr[0]); f[1] = to_frac<T>(fr[1]); f[2] = to_frac<T>(fr[2]);
      disp[0] += d[0]; disp[1] += d[1]; disp[2] += d[2];
      ok = valid_cell(i, j, k, p.nx, p.ny, p.nz);
    }
    P.ux[q] = u[0]; P.uy[q] = u[1]; P.uz[q] = u[2];
    if (!ok) {
      P.cell[q] = -1;
      atomicAdd(reinterpret_cast<unsigned long long*>(lost_ctr), 1ULL);
    } else {
      P.cell[q] = (int)cidx(i, j, k, p.nx, p.nxy);
      P.fx[q] = f[0]; P.fy[q] = f[1]; P.fz[q] = f[2];
      // rho^{n+3/2} at the end position
      deposit_cic(p, src, i, j, k, f[0], f[1], f[2], (T)0, (T)0, (T)0, p.qV);
      // J^{n+1} at the mid point: offset from the start cell in FP64
      double mf[3];
      const int mi = split_cell(i0, (double)f0x + 0.5 * disp[0], &mf[0]);
      const int mj = split_cell(j0, (double)f0y + 0.5 * disp[1], &mf[1]);
      const int mk = split_cell(k0, (double)f0z + 0.5 * disp[2], &mf[2]);
      deposit_cic(p, src, mi, mj, mk, to_frac<T>(mf[0]), to_frac<T>(mf[1]), to_frac<T>(mf[2]),
                  (T)(p.jfx * disp[0]), (T)(p.jfy * disp[1]), (T)(p.jfz * disp[2]), (T)0);
      kk = tile_key(p, i, j, k);
    }
  }
  key[q] = kk;
  rank[q] = bin_rank(count, kk);
}

// Host FP64 positions -> (cell, fraction) and the tile key; invalid
// positions mark the particle lost.
template <typename T, typename U>
__global__ void k_init_particles(PicP<T> p, long long np, const double* __restrict__ x,
                                 const double* __restrict__ y, const double* __restrict__ z,
                                 const double* __restrict__ ux, const double* __restrict__ uy,
                                 const double* __restrict__ uz, Parts<T, U> P,
                                 int* __restrict__ count, int* __restrict__ key,
                                 int* __restrict__ rank, long long* __restrict__ lost_ctr) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  double fr[3];
  const int i = split_cell(0, (x[q] - p.x0) / p.dxd, &fr[0]);
  const int j = split_cell(0, (y[q] - p.y0) / p.dyd, &fr[1]);
  const int k = split_cell(0, (z[q] - p.z0) / p.dzd, &fr[2]);
  int kk = p.nkeys;
  if (valid_cell(i, j, k, p.nx, p.ny, p.nz)) {
    P.cell[q] = (int)cidx(i, j, k, p.nx, p.nxy);
    kk = tile_key(p, i, j, k);
  } else {
    P.cell[q] = -1;
    atomicAdd(reinterpret_cast<unsigned long long*>(lost_ctr), 1ULL);
  }
  P.fx[q] = to_frac<T>(fr[0]); P.fy[q] = to_frac<T>(fr[1]); P.fz[q] = to_frac<T>(fr[2]);
  P.ux[q] = (U)ux[q]; P.uy[q] = (U)uy[q]; P.uz[q] = (U)uz[q];
  P.id[q] = (int)q;
  key[q] = kk;
  rank[q] = bin_rank(count, kk);
}

// rho of the particles at their present positions (initial rho^{1/2}).
template <typename T, typename U>
__global__ void k_deposit_rho(PicP<T> p, Parts<T, U> P, long long np, V4<T>* __restrict__ src) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const int cell = P.cell[q];
  if (cell < 0) return;
  const int i = cell % p.nx, j = (cell / p.nx) % p.ny, k = cell / (int)p.nxy;
  deposit_cic(p, src, i, j, k, P.fx[q], P.fy[q], P.fz[q], (T)0, (T)0, (T)0, p.qV);
}

// Exclusive scan of the per-tile counts (one block), resetting the counts for
// the next step.  offset[nkeys + 1] receives the total.  With advance != 0 the
// block also advances the step counter: it runs last in every step.
__global__ void __launch_bounds__(1024) k_scan_counts(int* __restrict__ count,
                                                      int* __restrict__ offset, int n,
                                                      StepState* __restrict__ st, int advance) {
  __shared__ int warp_sums[32];
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = min(n, (int)threadIdx.x * per), end = min(n, beg + per);
  int s = 0;
  for (int t = beg; t < end; ++t) s += count[t];
  // block-wide exclusive scan of s
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    warp_sums[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  int run = incl - s + (wid > 0 ? warp_sums[wid - 1] : 0);
  for (int t = beg; t < end; ++t) {
    const int c = count[t];
    offset[t] = run;
    run += c;
    count[t] = 0;
  }
  if (threadIdx.x == blockDim.x - 1) offset[n] = run;
  if (advance && threadIdx.x == 0) st->n += 1;
}

// Moves every particle to offset[key] + rank in the other buffer.
template <typename T, typename U>
__global__ void k_scatter(Parts<T, U> a, Parts<T, U> b, long long np, const int* __restrict__ key,
                          const int* __restrict__ rank, const int* __restrict__ offset) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const long long d = (long long)offset[key[q]] + rank[q];
  b.cell[d] = a.cell[q];
  b.fx[d] = a.fx[q]; b.fy[d] = a.fy[q]; b.fz[d] = a.fz[q];
  b.ux[d] = a.ux[q]; b.uy[d] = a.uy[q]; b.uz[d] = a.uz[q];
  b.id[d] = a.id[q];
}

// Copy-out in the original particle order: FP64 positions from (cell, f).
template <typename T, typename U>
__global__ void k_copy_out(PicP<T> p, Parts<T, U> P, long long np, double* __restrict__ out) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const long long d = P.id[q];
  const int cell = P.cell[q];
  double x = 0, y = 0, z = 0, lost = 1.0;
  if (cell >= 0) {
    const int i = cell % p.nx, j = (cell / p.nx) % p.ny, k = cell / (int)p.nxy;
    x = p.x0 + ((double)i + (double)P.fx[q]) * p.dxd;
    y = p.y0 + ((double)j + (double)P.fy[q]) * p.dyd;
    z = p.z0 + ((double)k + (double)P.fz[q]) * p.dzd;
    lost = 0.0;
  }
  out[0 * np + d] = x;
  out[1 * np + d] = y;
  out[2 * np + d] = z;
  out[3 * np + d] = (double)P.ux[q];
  out[4 * np + d] = (double)P.uy[q];
  out[5 * np + d] = (double)P.uz[q];
  out[6 * np + d] = lost;
}

}  // namespace mithra
