// field_kernels.cuh -- potential update (Eq. updateEquation) with the
// first-order Mur boundary (Sec. "First Order ABCs") fused in, E/B at the
// vertices (Sec. "Field Evaluation"), radiated power and field copy-out.
#pragma once
#include "common.cuh"

namespace mithra {

// Potential update of one interior cell c, all four components at once.
//   psi^{n+1} = -psi^{n-1} + a1 psi + a2 (bar_{i+1} + bar_{i-1})
//             + a4 (bar_{j+1} + bar_{j-1}) + a6 (psi_{k+1} + psi_{k-1}) + S
// with bar = A psi_{k-1} + (1 - 2A) psi_k + A psi_{k+1} (Eq. NSFDtrick) and
// S = (c dt)^2 (mu0 J, rho / eps0).
template <typename T>
__device__ inline V4<T> stencil_cell(const StencilP<T>& p, const V4<T>* __restrict__ cur,
                                     V4<T> pm, V4<T> s, long long c) {
  const long long nxy = p.nxy;
  const int nx = p.nx;
  auto bar = [&](long long q) {
    return p.A * (ldg4(cur + q - nxy) + ldg4(cur + q + nxy)) + p.omA2 * ldg4(cur + q);
  };
  V4<T> pc = ldg4(cur + c);
  V4<T> v = p.a1 * pc - pm;
  v = v + p.a2 * (bar(c + 1) + bar(c - 1));
  v = v + p.a4 * (bar(c + nx) + bar(c - nx));
  v = v + p.a6 * (ldg4(cur + c + nxy) + ldg4(cur + c - nxy));
  v = v + v4(p.sA * s.x, p.sA * s.y, p.sA * s.z, p.sphi * s.w);
  if (!p.space_charge) v.w = (T)0;
  return v;
}

// Mur update of the boundary vertices whose nearest interior vertex is c
// (i, j, k), using psi^{n+1}_c = pn and psi^{n-1}_c = pm before they are
// overwritten, and zero the boundary vertex's source.  For a boundary vertex b:
//   xi_b^{n+1} = b0 (xi_b^{n-1} + xi_c^{n+1}) + b1 (xi_b^n + xi_c^n) - xi_c^{n-1}
// with b0, b1 for the spacing d = |b - c| (face: the axis spacing; edge and
// corner: the diagonal).
template <typename T>
__device__ inline void mur_neighbours(const StencilP<T>& p, const V4<T>* __restrict__ cur,
                                      V4<T>* __restrict__ nxt, V4<T>* __restrict__ src, int i,
                                      int j, int k, long long c, V4<T> pn, V4<T> pm) {
  const int lo_x = (i == 1) ? -1 : 0, hi_x = (i == p.nx - 2) ? 1 : 0;
  const int lo_y = (j == 1) ? -1 : 0, hi_y = (j == p.ny - 2) ? 1 : 0;
  const int lo_z = (k == 1) ? -1 : 0, hi_z = (k == p.nz - 2) ? 1 : 0;
  if (!(lo_x | hi_x | lo_y | hi_y | lo_z | hi_z)) return;
  const V4<T> pcur = ldg4(cur + c);
  for (int dz = lo_z; dz <= hi_z; ++dz) {
    for (int dy = lo_y; dy <= hi_y; ++dy) {
      for (int dx = lo_x; dx <= hi_x; ++dx) {
        const int mask = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
        if (!mask) continue;
        const long long b = c + dx + (long long)dy * p.nx + (long long)dz * p.nxy;
        const V4<T> pbm = nxt[b];           // xi_b^{n-1}
        const V4<T> pb = ldg4(cur + b);     // xi_b^n
        V4<T> r = p.mb0[mask] * (pbm + pn) + p.mb1[mask] * (pb + pcur) - pm;
        if (!p.space_charge) r.w = (T)0;
        nxt[b] = r;
        src[b] = v4((T)0, (T)0, (T)0, (T)0);  // boundary sources are never used
      }
    }
  }
}

// One thread per vertex of the (x, y) plane, blocks marching nothing: the
// straightforward form.  lev[prev] holds psi^{n-1} on entry and psi^{n+1} on
// exit; the consumed sources are zeroed for the deposit of this step.
template <typename T>
__global__ void __launch_bounds__(256) k_potential_step(StencilP<T> p,
                                                        const V4<T>* __restrict__ cur,
                                                        V4<T>* __restrict__ nxt,
                                                        V4<T>* __restrict__ src) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i < 1 || i > p.nx - 2 || j < 1 || j > p.ny - 2 || k < 1 || k > p.nz - 2) return;
  const long long c = cidx(i, j, k, p.nx, p.nxy);
  const V4<T> pm = nxt[c];
  const V4<T> s = src[c];
  const V4<T> pn = stencil_cell(p, cur, pm, s, c);
  mur_neighbours(p, cur, nxt, src, i, j, k, c, pn, pm);
  nxt[c] = pn;
  src[c] = v4((T)0, (T)0, (T)0, (T)0);
}

// E and B at vertex v (interior) at t = (n+1/2) dt from level n (po) and
// level n+1 (pn):  B = (curl A^n + curl A^{n+1}) / 2,
// E = -(A^{n+1} - A^n) / dt - grad phi^n, central differences.
template <typename T>
__device__ inline void eb_vertex(const PicP<T>& p, const V4<T>* __restrict__ po,
                                 const V4<T>* __restrict__ pn, long long v, T E[3], T B[3]) {
  const long long nxy = p.nxy;
  const int nx = p.nx;
  const V4<T> o = ldg4(po + v), w = ldg4(pn + v);
  const V4<T> xp = ldg4(po + v + 1) + ldg4(pn + v + 1);
  const V4<T> xm = ldg4(po + v - 1) + ldg4(pn + v - 1);
  const V4<T> yp = ldg4(po + v + nx) + ldg4(pn + v + nx);
  const V4<T> ym = ldg4(po + v - nx) + ldg4(pn + v - nx);
  const V4<T> zp = ldg4(po + v + nxy) + ldg4(pn + v + nxy);
  const V4<T> zm = ldg4(po + v - nxy) + ldg4(pn + v - nxy);
  B[0] = (yp.z - ym.z) * p.inv4dy - (zp.y - zm.y) * p.inv4dz;
  B[1] = (zp.x - zm.x) * p.inv4dz - (xp.z - xm.z) * p.inv4dx;
  B[2] = (xp.y - xm.y) * p.inv4dx - (yp.x - ym.x) * p.inv4dy;
  // phi^n only: the level sums above include phi^{n+1}, so read phi^n apart
  const T phxp = ldg4(po + v + 1).w, phxm = ldg4(po + v - 1).w;
  const T phyp = ldg4(po + v + nx).w, phym = ldg4(po + v - nx).w;
  const T phzp = ldg4(po + v + nxy).w, phzm = ldg4(po + v - nxy).w;
  E[0] = -(w.x - o.x) * p.invdt - (phxp - phxm) * p.inv2dx;
  E[1] = -(w.y - o.y) * p.invdt - (phyp - phym) * p.inv2dy;
  E[2] = -(w.z - o.z) * p.invdt - (phzp - phzm) * p.inv2dz;
}

__device__ inline bool interior(int i, int j, int k, int nx, int ny, int nz) {
  return i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
}

// Whole-grid copy-out of one field (double), E/B evaluated on the fly.
// what: 0..2 E, 3..5 B, 6..9 component of lev (A_x, A_y, A_z, phi), 10..13
// component of src.
template <typename T>
__global__ void k_extract(PicP<T> p, const V4<T>* __restrict__ po, const V4<T>* __restrict__ pn,
                          const V4<T>* __restrict__ lev, const V4<T>* __restrict__ src, int what,
                          double* __restrict__ out) {
  const long long ncell = p.nxy * p.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double val = 0.0;
    if (what < 6) {
      const int i = (int)(c % p.nx);
      const int j = (int)((c / p.nx) % p.ny);
      const int k = (int)(c / p.nxy);
      if (interior(i, j, k, p.nx, p.ny, p.nz)) {
        T E[3], B[3];
        eb_vertex(p, po, pn, c, E, B);
        val = (double)(what < 3 ? E[what] : B[what - 3]);
      }
    } else {
      const V4<T> a = (what < 10) ? lev[c] : src[c];
      const int comp = (what - 6) & 3;
      val = (double)(comp == 0 ? a.x : comp == 1 ? a.y : comp == 2 ? a.z : a.w);
    }
    out[c] = val;
  }
}

// Host field -> one component of a device array.
template <typename T>
__global__ void k_insert(long long ncell, const double* __restrict__ in, V4<T>* __restrict__ dst,
                         int comp) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    T v = (T)in[c];
    V4<T> a = dst[c];
    if (comp == 0) a.x = v; else if (comp == 1) a.y = v; else if (comp == 2) a.z = v; else a.w = v;
    dst[c] = a;
  }
}

// Point samples: out[pt * m + s] for the s-th field of mask.
template <typename T>
__global__ void k_sample(PicP<T> p, const V4<T>* __restrict__ po, const V4<T>* __restrict__ pn,
                         const V4<T>* __restrict__ src, const int* __restrict__ ijk, long long npts,
                         unsigned mask, int m, double* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= npts) return;
  const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
  const long long c = cidx(i, j, k, p.nx, p.nxy);
  T E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
  if (interior(i, j, k, p.nx, p.ny, p.nz)) eb_vertex(p, po, pn, c, E, B);
  const V4<T> a = pn[c], s = src[c];
  const T vals[14] = {E[0], E[1], E[2], B[0], B[1], B[2], a.x, a.y, a.z, s.x, s.y, s.z, a.w, s.w};
  int slot = 0;
  for (int f = 0; f < 14; ++f)
    if (mask & (1u << f)) out[t * m + slot++] = (double)vals[f];
}

// Radiated power through vertex plane kp in the lab frame, FP64 accumulation:
// E'_x = g0 (E_x + b0 c B_y), E'_y = g0 (E_y - b0 c B_x),
// B'_x = g0 (B_x - b0 E_y / c), B'_y = g0 (B_y + b0 E_x / c),
// P = sum (E'_x B'_y - E'_y B'_x) / mu0 dx dy over interior (i, j).
// The result is added to *acc (zeroed by the caller); slot_from_state makes
// the kernel write into acc[state->n] (per-step recording) when below cap.
template <typename T>
__global__ void __launch_bounds__(256) k_power(PicP<T> p, const V4<T>* __restrict__ po,
                                               const V4<T>* __restrict__ pn, int kp, double g0,
                                               double b0, double* __restrict__ acc,
                                               const StepState* __restrict__ st, long long cap,
                                               int slot_from_state, int* __restrict__ err) {
  long long slot = 0;
  if (slot_from_state) {
    slot = st->n;
    if (slot >= cap) return;
  }
  const int nin = (p.nx - 2) * (p.ny - 2);
  double part = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nin; t += gridDim.x * blockDim.x) {
    const int i = 1 + t % (p.nx - 2);
    const int j = 1 + t / (p.nx - 2);
    T E[3], B[3];
    eb_vertex(p, po, pn, cidx(i, j, kp, p.nx, p.nxy), E, B);
    const double Ex = E[0], Ey = E[1], Bx = B[0], By = B[1];
    const double exl = g0 * (Ex + b0 * kC * By);
    const double eyl = g0 * (Ey - b0 * kC * Bx);
    const double bxl = g0 * (Bx - b0 * Ey / kC);
    const double byl = g0 * (By + b0 * Ex / kC);
    part += (exl * byl - eyl * bxl);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      v *= p.dxd * p.dyd / kMu0;
      if (!isfinite(v)) atomicOr(err, 1);
      atomicAdd(acc + slot, v);
    }
  }
}

}  // namespace mithra
