// field_kernels.cuh -- potential update (Eq. updateEquation) with the
// first-order Mur boundary (Sec. "First Order ABCs") fused in, E/B at the
// vertices (Sec. "Field Evaluation"), radiated power and field copy-out.
//
// Storage of the leapfrog: the newest level psi^{n+1} in one of two
// ping-pong arrays and the increment D = psi^{n+1} - psi^n in place.  The
// update equation is used in the algebraically equal increment form
//   D^{n+1/2} = D^{n-1/2} + (c dt)^2 lap_h psi^n + (c dt)^2 S,
//   psi^{n+1} = psi^n + D^{n+1/2},
// with the NSFD Laplacian written as sums of neighbour differences:
//   (c dt)^2 lap_h psi = rx^2 [A (DX_{k-1} + DX_{k+1}) + (1 - 2A) DX_k]
//                      + ry^2 [A (DY_{k-1} + DY_{k+1}) + (1 - 2A) DY_k]
//                      + rz^2 DZ,
// DX_k = (psi_{i+1,k} - psi_{i,k}) + (psi_{i-1,k} - psi_{i,k}) and likewise
// DY, DZ (r_l = c dt / d_l).  Expanding gives Eq. updateEquation's
// coefficients alpha'_1 .. alpha'_7.  In FP32 the rounding then scales with
// the increment rather than with the potential, so it no longer feeds the
// scheme's double root at omega = 0.
#pragma once
#include "common.cuh"
#include "tma.cuh"

namespace mithra {

template <typename T>
__device__ inline T mur_beta0(const StencilP<T>& p, int mask) {
  switch (mask) {
    case 1: return p.mb0[1];
    case 2: return p.mb0[2];
    case 3: return p.mb0[3];
    case 4: return p.mb0[4];
    case 5: return p.mb0[5];
    case 6: return p.mb0[6];
    default: return p.mb0[7];
  }
}

// Mur update of the boundary vertices whose nearest interior vertex is c
// (i, j, k).  With beta0 + beta1 = 1 the first-order condition
//   xi_b^{n+1} = b0 (xi_b^{n-1} + xi_c^{n+1}) + b1 (xi_b^n + xi_c^n) - xi_c^{n-1}
// becomes, in increments,  D_b^+ = b0 (D_c^+ - D_b^-) + D_c^-,
// b0 = (c dt - d)/(c dt + d) for d = |b - c| (face: the axis spacing; edge and
// corner: the diagonal).  Also zeroes the boundary vertex's source.
template <typename T>
__device__ inline void mur_neighbours(const StencilP<T>& p, const V4<T>* __restrict__ cur,
                                      V4<T>* __restrict__ nxt, V4<T>* __restrict__ D,
                                      V4<T>* __restrict__ src, int i, int j, int k,
                                      long long c, V4<T> dq_new, V4<T> dq_old) {
  const int lo_x = (i == 1) ? -1 : 0, hi_x = (i == p.nx - 2) ? 1 : 0;
  const int lo_y = (j == 1) ? -1 : 0, hi_y = (j == p.ny - 2) ? 1 : 0;
  const int lo_z = (k == 1) ? -1 : 0, hi_z = (k == p.nz - 2) ? 1 : 0;
  if (!(lo_x | hi_x | lo_y | hi_y | lo_z | hi_z)) return;
  for (int dz = lo_z; dz <= hi_z; ++dz) {
    for (int dy = lo_y; dy <= hi_y; ++dy) {
      for (int dx = lo_x; dx <= hi_x; ++dx) {
        const int mask = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
        if (!mask) continue;
        const long long b = c + dx + (long long)dy * p.nx + (long long)dz * p.nxy;
        const V4<T> db_old = D[b];
        V4<T> db = mur_beta0(p, mask) * (dq_new - db_old) + dq_old;
        if (!p.space_charge) db.w = (T)0;
        D[b] = db;
        nxt[b] = ldg4(cur + b) + db;
        src[b] = v4((T)0, (T)0, (T)0, (T)0);  // boundary sources are never used
      }
    }
  }
}

// Source term (c dt)^2 (mu0 J, rho / eps0).
template <typename T>
__device__ inline V4<T> source_term(const StencilP<T>& p, V4<T> s) {
  return v4(p.sA * s.x, p.sA * s.y, p.sA * s.z, p.sphi * s.w);
}

// Direct form: one thread per vertex, neighbours through L1.  cur holds
// psi^n, nxt receives psi^{n+1}, D is advanced in place; the consumed
// sources are zeroed for the deposit of this step.
template <typename T>
__global__ void __launch_bounds__(256) k_potential_step(StencilP<T> p,
                                                        const V4<T>* __restrict__ cur,
                                                        V4<T>* __restrict__ nxt,
                                                        V4<T>* __restrict__ D,
                                                        V4<T>* __restrict__ src) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i < 1 || i > p.nx - 2 || j < 1 || j > p.ny - 2 || k < 1 || k > p.nz - 2) return;
  const long long c = cidx(i, j, k, p.nx, p.nxy);
  const long long nxy = p.nxy;
  const int nx = p.nx;
  auto dsum = [&](long long q, long long off) {
    const V4<T> m = ldg4(cur + q);
    return (ldg4(cur + q + off) - m) + (ldg4(cur + q - off) - m);
  };
  const V4<T> pc = ldg4(cur + c);
  V4<T> L = p.rxA * (dsum(c - nxy, 1) + dsum(c + nxy, 1)) + p.rxB * dsum(c, 1);
  L = L + p.ryA * (dsum(c - nxy, nx) + dsum(c + nxy, nx)) + p.ryB * dsum(c, nx);
  L = L + p.rz2 * ((ldg4(cur + c + nxy) - pc) + (ldg4(cur + c - nxy) - pc));
  const V4<T> dm = D[c];
  V4<T> dp = dm + (L + source_term(p, src[c]));
  if (!p.space_charge) dp.w = (T)0;
  mur_neighbours(p, cur, nxt, D, src, i, j, k, c, dp, dm);
  D[c] = dp;
  nxt[c] = pc + dp;
  src[c] = v4((T)0, (T)0, (T)0, (T)0);
}

// ---------------------------------------------------------------------------
// Marching form of the same update.  A CTA owns a 32 x 8 column tile and a run
// of lz planes; it walks up in z.  For every plane three TMA box loads land in
// one stage of a shared-memory ring (kMStages stages in flight, one mbarrier
// each): psi^n of the tile plus a one-vertex halo, and the tile's D and
// sources.  A thread keeps, for its column and the planes k-1, k, k+1, the
// centre value and the x and y neighbour-difference sums in registers, so
// every input value is read from HBM about once and no thread waits on its
// own loads.  Stages are recycled through per-stage "empty" barriers that
// every warp arrives on, so warps do not wait for each other plane by plane.
// The Mur vertices are written by the thread of the adjacent interior vertex,
// as in the direct form.
constexpr int kMX = 32, kMY = 8, kMStages = 3;

template <typename T>
__host__ __device__ constexpr int march_psi_bytes() {
  return (kMX + 2) * (kMY + 2) * (int)sizeof(V4<T>);
}
template <typename T>
__host__ __device__ constexpr int march_col_bytes() {
  return kMX * kMY * (int)sizeof(V4<T>);
}
template <typename T>
__host__ __device__ constexpr int march_stage_bytes() {
  return ((march_psi_bytes<T>() + 127) / 128 * 128) + 2 * march_col_bytes<T>();
}
template <typename T>
__host__ __device__ constexpr int march_smem_bytes() {
  return kMStages * march_stage_bytes<T>() + 2 * kMStages * 8;
}

template <typename T>
__global__ void __launch_bounds__(kMX* kMY, (sizeof(T) == 4 ? 4 : 1)) k_potential_march(
    const __grid_constant__ CUtensorMap tm_cur, const __grid_constant__ CUtensorMap tm_d,
    const __grid_constant__ CUtensorMap tm_s, StencilP<T> p, const V4<T>* __restrict__ cur,
    V4<T>* __restrict__ nxt, V4<T>* __restrict__ D, V4<T>* __restrict__ src, int lz,
    int* __restrict__ err) {
  constexpr int HX = kMX + 2;
  constexpr int SB = march_stage_bytes<T>();
  constexpr int OFF_D = (march_psi_bytes<T>() + 127) / 128 * 128;
  constexpr int OFF_S = OFF_D + march_col_bytes<T>();
  constexpr int kWarps = kMX * kMY / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kMStages * SB);
  uint64_t* empty = full + kMStages;
  const int tx = threadIdx.x % kMX, ty = threadIdx.x / kMX;
  const int i0 = blockIdx.x * kMX, j0 = blockIdx.y * kMY;
  const int i = i0 + tx, j = j0 + ty;
  const int kb = max((int)blockIdx.z * lz, 1);
  const int ke = min((int)blockIdx.z * lz + lz, p.nz - 1);
  if (kb >= ke) return;             // uniform over the block
  const int nplanes = ke - kb + 2;  // psi^n planes kb-1 .. ke
  if (threadIdx.x == 0) {
    for (int s = 0; s < kMStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  // stage q holds psi^n of plane kb-1+q and, for interior planes, D and the
  // sources of plane kb-2+q (the plane updated when stage q arrives)
  auto issue = [&](int q) {
    const int s = q % kMStages;
    unsigned char* base = smem + s * SB;
    const int kd = kb - 2 + q;
    const bool cols = kd >= kb && kd < ke;
    mbar_arrive_expect_tx(&full[s], march_psi_bytes<T>() + (cols ? 2 * march_col_bytes<T>() : 0));
    tma_load_4d(base, &tm_cur, 0, i0 - 1, j0 - 1, kb - 1 + q, &full[s]);
    if (cols) {
      tma_load_4d(base + OFF_D, &tm_d, 0, i0, j0, kd, &full[s]);
      tma_load_4d(base + OFF_S, &tm_s, 0, i0, j0, kd, &full[s]);
    }
  };
  if (threadIdx.x == 0)
    for (int q = 0; q < kMStages && q < nplanes; ++q) issue(q);

  const bool active = i >= 1 && i <= p.nx - 2 && j >= 1 && j <= p.ny - 2;
  const int h = (ty + 1) * HX + (tx + 1);
  const V4<T> zero = v4((T)0, (T)0, (T)0, (T)0);
  // Reads stage q (centre, neighbour-difference sums, and D and the source of
  // the thread's own vertex); each warp then marks the stage consumed on its
  // empty barrier, and the issuing thread refills the slot with stage
  // q + kMStages once every warp has consumed it (no block-wide barrier).
  auto take = [&](int q, V4<T>& c, V4<T>& X, V4<T>& Y, V4<T>& dm, V4<T>& sv) {
    const int s = q % kMStages;
    const uint32_t par = (uint32_t)((q / kMStages) & 1);
    mbar_wait_bounded(&full[s], par, err);
    const unsigned char* base = smem + s * SB;
    const V4<T>* pl = reinterpret_cast<const V4<T>*>(base);
    c = pl[h];
    X = (pl[h + 1] - c) + (pl[h - 1] - c);
    Y = (pl[h + HX] - c) + (pl[h - HX] - c);
    if (q >= 2) {
      dm = reinterpret_cast<const V4<T>*>(base + OFF_D)[threadIdx.x];
      sv = reinterpret_cast<const V4<T>*>(base + OFF_S)[threadIdx.x];
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[s]);
    if (threadIdx.x == 0 && q + kMStages < nplanes) {
      mbar_wait_bounded(&empty[s], par, err);
      fence_proxy_async_smem();
      issue(q + kMStages);
    }
  };
  V4<T> cm, Xm, Ym, c0, X0, Y0, cp, Xp, Yp, dm = zero, sv = zero;
  take(0, cm, Xm, Ym, dm, sv);
  take(1, c0, X0, Y0, dm, sv);
  const long long col = (long long)j * p.nx + i;
  for (int k = kb; k < ke; ++k) {
    take(k - kb + 2, cp, Xp, Yp, dm, sv);
    if (active) {
      V4<T> L = p.rxA * (Xm + Xp) + p.rxB * X0;
      L = L + p.ryA * (Ym + Yp) + p.ryB * Y0;
      L = L + p.rz2 * ((cp - c0) + (cm - c0));
      V4<T> dp = dm + (L + source_term(p, sv));
      if (!p.space_charge) dp.w = (T)0;
      const long long c = (long long)k * p.nxy + col;
      mur_neighbours(p, cur, nxt, D, src, i, j, k, c, dp, dm);
      D[c] = dp;
      nxt[c] = c0 + dp;
      src[c] = zero;
    }
    cm = c0; Xm = X0; Ym = Y0;
    c0 = cp; X0 = Xp; Y0 = Yp;
  }
}

// E and B at vertex v (interior) at t = (n+1/2) dt from psi^{n+1} (pn) and
// the increment D = psi^{n+1} - psi^n:  B = (curl A^n + curl A^{n+1}) / 2 is
// the curl of the mid level pn - D/2; E = -D_A / dt - grad phi^n with
// phi^n = pn.w - D.w; central differences.
template <typename T>
__device__ inline void eb_vertex(const PicP<T>& p, const V4<T>* __restrict__ pn,
                                 const V4<T>* __restrict__ D, long long v, T E[3], T B[3]) {
  const long long nxy = p.nxy;
  const int nx = p.nx;
  const T half = (T)0.5;
  auto mid = [&](long long q) {
    const V4<T> a = ldg4(pn + q), d = ldg4(D + q);
    return v4(a.x - half * d.x, a.y - half * d.y, a.z - half * d.z, a.w - d.w);
  };
  // .w of mid() is phi^n
  const V4<T> xp = mid(v + 1), xm = mid(v - 1);
  const V4<T> yp = mid(v + nx), ym = mid(v - nx);
  const V4<T> zp = mid(v + nxy), zm = mid(v - nxy);
  const V4<T> dc = ldg4(D + v);
  B[0] = (yp.z - ym.z) * p.inv2dy - (zp.y - zm.y) * p.inv2dz;
  B[1] = (zp.x - zm.x) * p.inv2dz - (xp.z - xm.z) * p.inv2dx;
  B[2] = (xp.y - xm.y) * p.inv2dx - (yp.x - ym.x) * p.inv2dy;
  E[0] = -dc.x * p.invdt - (xp.w - xm.w) * p.inv2dx;
  E[1] = -dc.y * p.invdt - (yp.w - ym.w) * p.inv2dy;
  E[2] = -dc.z * p.invdt - (zp.w - zm.w) * p.inv2dz;
}

__device__ inline bool interior(int i, int j, int k, int nx, int ny, int nz) {
  return i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
}

// Whole-grid copy-out of one field (double), E/B evaluated on the fly.
// what: 0..2 E, 3..5 B, 6..9 component of lev (A_x, A_y, A_z, phi), 10..13
// component of src.
template <typename T>
__global__ void k_extract(PicP<T> p, const V4<T>* __restrict__ pn, const V4<T>* __restrict__ D,
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
        eb_vertex(p, pn, D, c, E, B);
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

// D = newest - previous level (after a level was set from the host).
template <typename T>
__global__ void k_increment(long long ncell, const V4<T>* __restrict__ pn,
                            const V4<T>* __restrict__ po, V4<T>* __restrict__ D) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x)
    D[c] = pn[c] - po[c];
}

// Point samples: out[pt * m + s] for the s-th field of mask.
template <typename T>
__global__ void k_sample(PicP<T> p, const V4<T>* __restrict__ pn, const V4<T>* __restrict__ D,
                         const V4<T>* __restrict__ src, const int* __restrict__ ijk, long long npts,
                         unsigned mask, int m, double* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= npts) return;
  const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
  const long long c = cidx(i, j, k, p.nx, p.nxy);
  T E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
  if (interior(i, j, k, p.nx, p.ny, p.nz)) eb_vertex(p, pn, D, c, E, B);
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
__global__ void __launch_bounds__(256) k_power(PicP<T> p, const V4<T>* __restrict__ pn,
                                               const V4<T>* __restrict__ D, int kp, double g0,
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
    eb_vertex(p, pn, D, cidx(i, j, kp, p.nx, p.nxy), E, B);
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
