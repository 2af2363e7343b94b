// field_kernels.cuh -- potential update (Eq. updateEquation) with the Mur
// boundary (Sec. "First Order ABCs", "Second Order ABCs": its own kernel, and
// first-order Mur at the x faces inside the z-marching update), E/B at the
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

// Second-order Mur (Sec. "Second Order ABCs") at the face vertex b next to
// interior vertex c, face normal to the single axis of mask: the printed
// update equals the first-order one (beta1 = 1 - beta0 on xi^n) plus
//   sum_t g_t [(d^2_t xi^n)_b + (d^2_t xi^n)_c],  d^2_t f = f_{t+} - 2 f + f_{t-},
// over the two tangential axes t, g_t = (c dt/d_t)^2 d_a / (2 (c dt + d_a)),
// which is the increment to add to the first-order D_b.
template <typename T>
__device__ inline V4<T> mur2_terms(const StencilP<T>& p, const V4<T>* __restrict__ cur, int mask,
                                   long long b, long long c) {
  const int a = mask == 1 ? 0 : (mask == 2 ? 1 : 2);
  const long long o1 = (a == 0) ? (long long)p.nx : 1;
  const long long o2 = (a == 2) ? (long long)p.nx : p.nxy;
  auto d2 = [&](long long v, long long o) {
    const V4<T> m = ldg4(cur + v);
    return (ldg4(cur + v + o) - m) + (ldg4(cur + v - o) - m);
  };
  // coefficients picked without a run-time index into the parameter block
  const T g1 = a == 0 ? p.m2[0][0] : (a == 1 ? p.m2[1][0] : p.m2[2][0]);
  const T g2 = a == 0 ? p.m2[0][1] : (a == 1 ? p.m2[1][1] : p.m2[2][1]);
  return g1 * (d2(b, o1) + d2(c, o1)) + g2 * (d2(b, o2) + d2(c, o2));
}

// A source vertex needs its zeroing store only when the last deposit touched
// it (the bunch covers a small part of the grid; NaN counts as touched).
template <typename T>
__device__ inline bool nonzero(V4<T> s) {
  return !(s.x == (T)0 && s.y == (T)0 && s.z == (T)0 && s.w == (T)0);
}

// Source term (c dt)^2 (mu0 J, rho / eps0).
template <typename T>
__device__ inline V4<T> source_term(const StencilP<T>& p, V4<T> s) {
  return v4(p.sA * s.x, p.sA * s.y, p.sA * s.z, p.sphi * s.w);
}

// The new increment D^{n+1/2} = D^{n-1/2} + (L + source term), L the
// (c dt)^2-scaled Laplacian (the form every kernel of the register
// z-marching family uses; kPack as in vadd).
template <bool kPack, typename T>
__device__ inline V4<T> next_increment(const StencilP<T>& p, V4<T> dm, V4<T> L, V4<T> s) {
  return vadd<kPack>(dm, vfma4<kPack>(v4(p.sA, p.sA, p.sA, p.sphi), s, L));
}

// (c dt)^2 lap_h of the level read by ld at interior vertex c, the direct
// form: neighbours of psi^n read through L1.  With compensated levels (kLo)
// the Laplacian is taken of both parts, hi and lo: the neighbour differences
// of hi are exact or nearly so, so the sum carries the level to about twice
// FP32's precision.
template <typename T, typename Load>
__device__ inline V4<T> laplacian(const StencilP<T>& p, Load&& ld, long long c) {
  const long long nxy = p.nxy;
  const int nx = p.nx;
  auto dsum = [&](long long q, long long off) {
    const V4<T> m = ld(q);
    return (ld(q + off) - m) + (ld(q - off) - m);
  };
  const V4<T> ac = ld(c);
  V4<T> L = p.rxA * (dsum(c - nxy, 1) + dsum(c + nxy, 1)) + p.rxB * dsum(c, 1);
  L = L + p.ryA * (dsum(c - nxy, nx) + dsum(c + nxy, nx)) + p.ryB * dsum(c, nx);
  return L + p.rz2 * ((ld(c + nxy) - ac) + (ld(c - nxy) - ac));
}

// Register z-marching form of the interior update (no shared memory): a
// thread owns column (i, j) for a run of lz planes and keeps, for the planes
// k-1 and k, what they bring to the Laplacian (PlaneTerms) in registers, so a
// plane of psi^n is read once per run (its x and y neighbours are the
// adjacent threads' loads and hit L1) instead of three times as in the
// direct form.  The same sums as the direct form, grouped per plane.
template <typename T>
struct PlaneSums {
  V4<T> c, X, Y;
};

template <bool kPack, typename T, typename Load>
__device__ inline PlaneSums<T> plane_sums(Load&& ld, long long q, int nx) {
  PlaneSums<T> r;
  r.c = ld(q);
  r.X = vadd<kPack>(vsub<kPack>(ld(q + 1), r.c), vsub<kPack>(ld(q - 1), r.c));
  r.Y = vadd<kPack>(vsub<kPack>(ld(q + nx), r.c), vsub<kPack>(ld(q - nx), r.c));
  return r;
}

template <typename T>
__device__ inline V4<T> plane_laplacian(const StencilP<T>& p, const PlaneSums<T>& m,
                                        const PlaneSums<T>& z, const PlaneSums<T>& pl) {
  V4<T> L = p.rxA * (m.X + pl.X) + p.rxB * z.X;
  L = L + p.ryA * (m.Y + pl.Y) + p.ryB * z.Y;
  return L + p.rz2 * ((pl.c - z.c) + (m.c - z.c));
}

// What one plane brings to the NSFD Laplacian (Eq. NSFDCoefficient) at its
// own column and its z neighbours': a = rxA X + ryA Y (as plane k-1 or k+1),
// b = rxB X + ryB Y (as plane k), X and Y the x and y neighbour-difference
// sums of the level (hi + lo parts: the sums are small, so merging the parts
// there costs nothing), and the level at the column, hi c and lo cl, for the
// z second difference, formed part by part.  The z-marching loop carries
// two planes of these instead of two planes of hi and lo sums each.  The
// plain levels' arithmetic runs on packed FP32 pairs (kPack); the
// compensated levels' stays component-wise (packed, the compensated kernel
// ran 3 % slower at its register cap, the plain one 2 % faster).
template <typename T>
struct PlaneTerms {
  V4<T> a, b, c, cl;
};

template <bool kLo, typename T, typename LdHi, typename LdLo>
__device__ inline PlaneTerms<T> plane_terms(const StencilP<T>& p, LdHi&& hi, LdLo&& lo,
                                            long long q, int nx) {
  constexpr bool kPack = !kLo;
  const PlaneSums<T> h = plane_sums<kPack, T>(hi, q, nx);
  V4<T> X = h.X, Y = h.Y, cl = v4((T)0, (T)0, (T)0, (T)0);
  if (kLo) {
    const PlaneSums<T> l = plane_sums<kPack, T>(lo, q, nx);
    X = X + l.X;
    Y = Y + l.Y;
    cl = l.c;
  }
  return {vfma<kPack>(p.rxA, X, vmul<kPack>(p.ryA, Y)),
          vfma<kPack>(p.rxB, X, vmul<kPack>(p.ryB, Y)), h.c, cl};
}

// (The sum (m.a + z.b) + pl.a in this order: the z-marching loop carries
// its first part from one plane to the next.)
template <bool kLo, typename T>
__device__ inline V4<T> terms_laplacian(const StencilP<T>& p, const PlaneTerms<T>& m,
                                        const PlaneTerms<T>& z, const PlaneTerms<T>& pl) {
  constexpr bool kPack = !kLo;
  V4<T> L = vfma<kPack>(p.rz2, vadd<kPack>(vsub<kPack>(pl.c, z.c), vsub<kPack>(m.c, z.c)),
                        vadd<kPack>(vadd<kPack>(m.a, z.b), pl.a));
  if (kLo) L = L + p.rz2 * ((pl.cl - z.cl) + (m.cl - z.cl));
  return L;
}

// D^{n+1/2} at interior vertex c (and D^{n-1/2}, the source there): the
// Laplacian in the direct form's order, or with kTerms in the z-marching
// form's (so that a boundary kernel beside that form sees its increments bit
// for bit).
template <bool kLo, typename T, bool kTerms = false>
__device__ inline V4<T> interior_increment(const StencilP<T>& p, const V4<T>* __restrict__ cur,
                                           const LoV4* __restrict__ curlo,
                                           const V4<T>* __restrict__ D,
                                           const V4<T>* __restrict__ src, long long c,
                                           V4<T>* dm_out, V4<T>* sv_out) {
  auto hi = [&](long long q) { return ldg4(cur + q); };
  auto lo = [&](long long q) { return ld_lo<T>(curlo, q); };
  V4<T> L;
  if (kTerms) {  // the arithmetic of the z-marching form, term for term
    const int nx = p.nx;
    L = terms_laplacian<kLo>(p, plane_terms<kLo>(p, hi, lo, c - p.nxy, nx),
                             plane_terms<kLo>(p, hi, lo, c, nx),
                             plane_terms<kLo>(p, hi, lo, c + p.nxy, nx));
  } else {
    L = laplacian(p, hi, c);
    if (kLo) L = L + laplacian(p, lo, c);
  }
  const V4<T> dm = D[c];
  const V4<T> sv = src[c];
  V4<T> dp = kTerms ? next_increment<!kLo>(p, dm, L, sv) : dm + (L + source_term(p, sv));
  if (!p.space_charge) dp.w = (T)0;
  *dm_out = dm;
  *sv_out = sv;
  return dp;
}

// (hi, lo) + d for each component: Knuth's TwoSum of hi and d, its error
// added to lo, then the pair renormalised (Dekker's FastTwoSum), so that hi
// stays the nearest float of the level.
template <typename T>
__device__ inline void comp_add1(T hi, T lo, T d, T* ho, T* lout) {
  const T s = hi + d;
  const T bb = s - hi;
  const T err = (hi - (s - bb)) + (d - bb);
  const T l = lo + err;
  const T h = s + l;
  *ho = h;
  *lout = l - (h - s);
}

template <typename T>
__device__ inline void comp_add(V4<T> hi, V4<T> lo, V4<T> d, V4<T>* ho, V4<T>* lout) {
  comp_add1(hi.x, lo.x, d.x, &ho->x, &lout->x);
  comp_add1(hi.y, lo.y, d.y, &ho->y, &lout->y);
  comp_add1(hi.z, lo.z, d.z, &ho->z, &lout->z);
  comp_add1(hi.w, lo.w, d.w, &ho->w, &lout->w);
}

// psi^{n+1} = psi^n + D^{n+1/2} at vertex c, compensated or plain.
template <bool kLo, typename T>
__device__ inline void store_level(const V4<T>* __restrict__ cur, const LoV4* __restrict__ curlo,
                                   V4<T>* __restrict__ nxt, LoV4* __restrict__ nxtlo,
                                   long long c, V4<T> d) {
  if (kLo) {
    V4<T> h, l;
    comp_add(ldg4(cur + c), ld_lo<T>(curlo, c), d, &h, &l);
    nxt[c] = h;
    st_lo(nxtlo, c, l);
  } else {
    nxt[c] = ldg4(cur + c) + d;
  }
}

// Boundary vertex b of the launch shape below: grid (x, y, 6) of 32 x 8
// blocks, blockIdx.z picks the face (z-, z+: all (i, j); y-, y+: all i, k in
// [1, nz-2]; x-, x+: j, k in [1, ny-2] x [1, nz-2]), the block's 2-D thread
// index the vertex on it.  Returns false for threads past the face.
__device__ inline bool boundary_vertex(int nx, int ny, int nz, int* i, int* j, int* k) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  const int f = blockIdx.z;
  if (f < 2) {
    if (u >= nx || v >= ny) return false;
    *i = u; *j = v; *k = f == 0 ? 0 : nz - 1;
  } else if (f < 4) {
    if (u >= nx || v >= nz - 2) return false;
    *i = u; *k = v + 1; *j = f == 2 ? 0 : ny - 1;
  } else {
    if (u >= ny - 2 || v >= nz - 2) return false;
    *j = u + 1; *k = v + 1; *i = f == 4 ? 0 : nx - 1;
  }
  return true;
}

// Mur update of every boundary vertex b, launched before the interior
// update (which then carries no boundary code).  With beta0 + beta1 = 1 the
// first-order condition
//   xi_b^{n+1} = b0 (xi_b^{n-1} + xi_q^{n+1}) + b1 (xi_b^n + xi_q^n) - xi_q^{n-1}
// becomes, in increments,  D_b^+ = b0 (D_q^+ - D_b^-) + D_q^-,
// for q the nearest interior vertex and b0 = (c dt - d)/(c dt + d), d = |b - q|
// (face: the axis spacing; edge and corner: the diagonal).  D_q^+ is
// evaluated here from the same inputs as the interior update (whose D_q^- is
// still in place).  Face vertices of a second-order grid add mur2_terms.  The
// boundary sources are zeroed (no deposit reads them).
// Whether the x+ face's lanes share a warp with their interior neighbours
// (blocks are 32 wide along x, so i = nx-1 is a warp's lane 0 when
// (nx-1) % 32 == 0).
__host__ __device__ inline bool xhi_fused(int nx) { return ((nx - 1) & 31) != 0; }

// The boundary vertices that k_potential_zloop_mur1 leaves, one per thread
// of a 1-D grid of rest_count threads: the z faces, the y faces (edges
// included), and the x+ face when its lanes cannot share a warp with their
// neighbours (xhi_fused false).
__host__ __device__ inline long long rest_count(int nx, int ny, int nz) {
  return 2LL * nx * ny + 2LL * nx * (nz - 2) +
         (xhi_fused(nx) ? 0LL : (long long)(ny - 2) * (nz - 2));
}
__device__ inline bool rest_vertex_at(long long t, int nx, int ny, int nz, int* i, int* j,
                                      int* k) {
  const long long nxy = (long long)nx * ny;
  if (t < 2 * nxy) {  // z faces
    const long long r = t % nxy;
    *i = (int)(r % nx); *j = (int)(r / nx); *k = t < nxy ? 0 : nz - 1;
    return true;
  }
  t -= 2 * nxy;
  const long long ny_face = (long long)nx * (nz - 2);
  if (t < 2 * ny_face) {  // y faces, planes 1 .. nz-2
    const long long r = t % ny_face;
    *i = (int)(r % nx); *k = 1 + (int)(r / nx); *j = t < ny_face ? 0 : ny - 1;
    return true;
  }
  t -= 2 * ny_face;
  if (!xhi_fused(nx) && t < (long long)(ny - 2) * (nz - 2)) {  // x+ face
    *i = nx - 1; *j = 1 + (int)(t % (ny - 2)); *k = 1 + (int)(t / (ny - 2));
    return true;
  }
  return false;
}

__device__ inline bool rest_vertex(int nx, int ny, int nz, int* i, int* j, int* k) {
  return rest_vertex_at(blockIdx.x * (long long)blockDim.x + threadIdx.x, nx, ny, nz, i, j, k);
}

// Mur update of boundary vertex (i, j, k) (see k_mur_boundary).
template <bool kLo, typename T, bool kTerms>
__device__ __forceinline__ void mur_vertex(const StencilP<T>& p, const V4<T>* __restrict__ cur,
                                           const LoV4* __restrict__ curlo,
                                           V4<T>* __restrict__ nxt, LoV4* __restrict__ nxtlo,
                                           V4<T>* __restrict__ D, V4<T>* __restrict__ src, int i,
                                           int j, int k) {
  const int qi = min(max(i, 1), p.nx - 2), qj = min(max(j, 1), p.ny - 2),
            qk = min(max(k, 1), p.nz - 2);
  const int mask = (qi != i) | ((qj != j) << 1) | ((qk != k) << 2);
  const long long b = cidx(i, j, k, p.nx, p.nxy), q = cidx(qi, qj, qk, p.nx, p.nxy);
  V4<T> dq_old, sq;
  const V4<T> dq_new = interior_increment<kLo, T, kTerms>(p, cur, curlo, D, src, q, &dq_old, &sq);
  const V4<T> db_old = D[b];
  V4<T> db = mur_beta0(p, mask) * (dq_new - db_old) + dq_old;
  if (p.mur2 && (mask & (mask - 1)) == 0) db = db + mur2_terms(p, cur, mask, b, q);
  if (!p.space_charge) db.w = (T)0;
  D[b] = db;
  store_level<kLo>(cur, curlo, nxt, nxtlo, b, db);
  src[b] = v4((T)0, (T)0, (T)0, (T)0);
}

// With kRest, only the vertices of rest_vertex (1-D launch of rest_count
// threads).  kTerms: the interior update is the z-marching form, whose
// arithmetic D_q^+ is recomputed with.
template <bool kLo, typename T, bool kRest = false, bool kTerms = false>
__global__ void __launch_bounds__(256) k_mur_boundary(StencilP<T> p,
                                                      const V4<T>* __restrict__ cur,
                                                      const LoV4* __restrict__ curlo,
                                                      V4<T>* __restrict__ nxt,
                                                      LoV4* __restrict__ nxtlo,
                                                      V4<T>* __restrict__ D,
                                                      V4<T>* __restrict__ src) {
  int i, j, k;
  if (kRest ? !rest_vertex(p.nx, p.ny, p.nz, &i, &j, &k)
            : !boundary_vertex(p.nx, p.ny, p.nz, &i, &j, &k))
    return;
  mur_vertex<kLo, T, kTerms>(p, cur, curlo, nxt, nxtlo, D, src, i, j, k);
}

// Launch shape of k_mur_boundary.
__host__ inline dim3 mur_grid(int nx, int ny, int nz) {
  const int d0 = nx > ny ? nx : ny;
  const int d1 = ny > nz ? ny : nz;
  return dim3((d0 + 31) / 32, (d1 + 7) / 8, 6);
}

// Direct form of the interior update: one thread per vertex, neighbours
// through L1.  cur holds psi^n, nxt receives psi^{n+1}, D is advanced in
// place; the consumed sources are zeroed for the deposit of this step
// (stored only where non-zero).
template <bool kLo, typename T>
__global__ void __launch_bounds__(256) k_potential_step(StencilP<T> p,
                                                        const V4<T>* __restrict__ cur,
                                                        const LoV4* __restrict__ curlo,
                                                        V4<T>* __restrict__ nxt,
                                                        LoV4* __restrict__ nxtlo,
                                                        V4<T>* __restrict__ D,
                                                        V4<T>* __restrict__ src) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i < 1 || i > p.nx - 2 || j < 1 || j > p.ny - 2 || k < 1 || k > p.nz - 2) return;
  const long long c = cidx(i, j, k, p.nx, p.nxy);
  V4<T> dm, sv;
  const V4<T> dp = interior_increment<kLo>(p, cur, curlo, D, src, c, &dm, &sv);
  if (nonzero(sv)) src[c] = v4((T)0, (T)0, (T)0, (T)0);
  D[c] = dp;
  store_level<kLo>(cur, curlo, nxt, nxtlo, c, dp);
}


// kMur: the lanes of the x faces (i = 0, and i = nx-1 when xhi_fused) run
// the column loop on their own boundary vertex b and, instead of the
// interior update, take first-order Mur (the condition of k_mur_boundary)
// from the increments D_q^-, D_q^+ of the neighbouring lane's vertex q, read
// by warp shuffle: D_b^+ = b0 (D_q^+ - D_b^-) + D_q^-.  Their loads fall in
// the rows the warp reads anyway; every other boundary vertex is left to
// k_mur_boundary<.., kRest = true>.
template <bool kLo, typename T, bool kMur>
__device__ __forceinline__ void zloop_body(const StencilP<T>& p, const V4<T>* __restrict__ cur,
                                           const LoV4* __restrict__ curlo,
                                           V4<T>* __restrict__ nxt, LoV4* __restrict__ nxtlo,
                                           V4<T>* __restrict__ D, V4<T>* __restrict__ src,
                                           int lz, int bx, int by, int bz) {
  const int i = bx * 32 + threadIdx.x;
  const int j = by * 8 + threadIdx.y;
  const int kb = max(bz * lz, 1);
  const int ke = min(bz * lz + lz, p.nz - 1);
  const bool xb = kMur && (i == 0 || (i == p.nx - 1 && xhi_fused(p.nx)));
  const bool active = kb < ke && j >= 1 && j <= p.ny - 2 && ((i >= 1 && i <= p.nx - 2) || xb);
  unsigned live = 0;
  if (kMur) live = __ballot_sync(0xffffffffu, active);
  if (!active) return;
  bool xwarp = false;
  int from = 0;
  if (kMur) {
    xwarp = __any_sync(live, xb);
    const int lane = threadIdx.x & 31;
    from = i == 0 ? lane + 1 : (xb ? lane - 1 : lane);
  }
  const long long col = (long long)j * p.nx + i;
  const int nx = p.nx;
  auto hi = [&](long long q) { return ldg4(cur + q); };
  auto lo = [&](long long q) { return ld_lo<T>(curlo, q); };
  // the loop carries m.a + z.b (ab), z.a and the column's hi and lo of the
  // planes k-1 and k: a plane's b term is used only while it is plane k,
  // so 24 instead of 32 values (measured 2 % off the compensated update)
  V4<T> ab, a0, cm, clm, c0, cl0;
  {
    const PlaneTerms<T> tm = plane_terms<kLo>(p, hi, lo, (long long)(kb - 1) * p.nxy + col, nx);
    const PlaneTerms<T> t0 = plane_terms<kLo>(p, hi, lo, (long long)kb * p.nxy + col, nx);
    ab = vadd<!kLo>(tm.a, t0.b);
    a0 = t0.a;
    cm = tm.c; clm = tm.cl; c0 = t0.c; cl0 = t0.cl;
  }
  // sources: loaded (and cleared) in the tiles the particle step marked only
  const bool src_every = p.dirty == nullptr || *p.src_all != 0;
  const int trow = (j >> 3) * p.ntx + (i >> 3), ntxy = p.ntx * p.nty;
  // one lane a 128-byte line asks L2 for the level row two planes ahead and
  // the increment row one plane ahead while this plane is updated: the
  // loads of an iteration alone keep too few bytes in flight to cover the
  // DRAM latency (measured: 7 % off the FP32 update, 4 % off the
  // compensated one; prefetching the lo parts as well cost more than it
  // saved)
  constexpr int kPerLine = 128 / (int)sizeof(V4<T>);
  const bool pf_lane = (threadIdx.x % kPerLine) == 0;
  for (int k = kb; k < ke; ++k) {
    const long long q = (long long)k * p.nxy + col;
    if (pf_lane && k + 2 < p.nz) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(cur + q + 2 * p.nxy));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(D + q + p.nxy));
    }
    const PlaneTerms<T> tp = plane_terms<kLo>(p, hi, lo, q + p.nxy, nx);
    // terms_laplacian's arithmetic with m.a + z.b carried
    V4<T> L = vfma<!kLo>(p.rz2, vadd<!kLo>(vsub<!kLo>(tp.c, c0), vsub<!kLo>(cm, c0)),
                         vadd<!kLo>(ab, tp.a));
    if (kLo) L = L + p.rz2 * ((tp.cl - cl0) + (clm - cl0));
    const V4<T> dm = D[q];
    V4<T> sv = v4((T)0, (T)0, (T)0, (T)0);
    if (src_every || p.dirty[(k >> 3) * ntxy + trow] != 0) sv = src[q];
    V4<T> dp = next_increment<!kLo>(p, dm, L, sv);
    if (kMur && xwarp) {  // warp-uniform
      const V4<T> dq = v4(__shfl_sync(live, dp.x, from), __shfl_sync(live, dp.y, from),
                          __shfl_sync(live, dp.z, from), __shfl_sync(live, dp.w, from));
      const V4<T> mq = v4(__shfl_sync(live, dm.x, from), __shfl_sync(live, dm.y, from),
                          __shfl_sync(live, dm.z, from), __shfl_sync(live, dm.w, from));
      if (xb) dp = mur_beta0(p, 1) * (dq - dm) + mq;
    }
    if (!p.space_charge) dp.w = (T)0;
    if (nonzero(sv)) src[q] = v4((T)0, (T)0, (T)0, (T)0);
    D[q] = dp;
    if (kLo) {
      V4<T> h, l;
      comp_add(c0, cl0, dp, &h, &l);
      nxt[q] = h;
      st_lo(nxtlo, q, l);
    } else {
      nxt[q] = vadd<true>(c0, dp);
    }
    ab = vadd<!kLo>(a0, tp.b);
    a0 = tp.a;
    cm = c0; clm = cl0; c0 = tp.c; cl0 = tp.cl;
  }
}

template <bool kLo, typename T>
__global__ void __launch_bounds__(256) k_potential_zloop(StencilP<T> p,
                                                         const V4<T>* __restrict__ cur,
                                                         const LoV4* __restrict__ curlo,
                                                         V4<T>* __restrict__ nxt,
                                                         LoV4* __restrict__ nxtlo,
                                                         V4<T>* __restrict__ D,
                                                         V4<T>* __restrict__ src, int lz) {
  zloop_body<kLo, T, false>(p, cur, curlo, nxt, nxtlo, D, src, lz, blockIdx.x, blockIdx.y,
                            blockIdx.z);
}

// The same with first-order Mur fused; the register caps keep the
// occupancy of the plain form.
template <bool kLo, typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (kLo ? 3 : 4) : (kLo ? 1 : 2))
    k_potential_zloop_mur1(StencilP<T> p, const V4<T>* __restrict__ cur,
                           const LoV4* __restrict__ curlo, V4<T>* __restrict__ nxt,
                           LoV4* __restrict__ nxtlo, V4<T>* __restrict__ D,
                           V4<T>* __restrict__ src, int lz) {
  zloop_body<kLo, T, true>(p, cur, curlo, nxt, nxtlo, D, src, lz, blockIdx.x, blockIdx.y,
                           blockIdx.z);
}

// Seed field (Sec. "Seed Field"): a plane wave (this kernel) or a Gaussian
// beam (k_seed_tfsf_beam below) along z, given in the lab like the optical
// undulator, injected by the total-field/scattered-field planes
// k = 2 (last scattered-field plane, next to the z = z_min boundary) and
// k = 3 (first total-field plane).  The update of level n+1 took, across the
// two planes, neighbours of the other region; with the incident vector
// potential f^n uniform in x and y, the coupling of a plane to its z
// neighbour is (c dt/dz)^2 f (the NSFD cross terms of a uniform field sum to
// the same), so the increment and level n+1 get
//   k = 2:  -(c dt/dz)^2 f^n(z_3),    k = 3:  +(c dt/dz)^2 f^n(z_2)
// in the A_x, A_y components (the seed has no phi and no A_z).
struct SeedP {
  int on, signal;
  double ax, ay;                  // A0 times the unit polarization
  double w0, cep, t0o, inv_tv, env_a;
  double tau_t, tau_z, tau_c;     // tau = tau_t t + tau_z z + tau_c
  double z2, z3;                  // rest-frame z of the planes k = 2 and 3
  double t0, dt;
  // Gaussian beam (beam = 1)
  int beam;
  double px, py;                  // unit polarization
  double xf, yf;                  // transverse position of the focus
  double zeta_t, zeta_z, zeta_c;  // zeta = zeta_t t + zeta_z z + zeta_c, past the focus
  double zr_p, zr_q;              // Rayleigh lengths along and across p
  double inv_w2p, inv_w2q;        // 1 / waist^2 along and across p
  double gx0, gy0, gdx, gdy;      // vertex x = gx0 + i gdx, y = gy0 + j gdy
  double kxA, kyA, kz2;           // (c dt/dx)^2 A, (c dt/dy)^2 A, (c dt/dz)^2
};

// Signal s(x) of the FIELD section's list (see mithra_undulator), FP64,
// with the carrier phase cep + ph.
__device__ inline double seed_signal(const SeedP& q, double x, double ph = 0.0) {
  const double C = cos(q.w0 * x + q.cep + ph);
  switch (q.signal) {
    case 0: return -4.0 * 0.69314718055994531 * (x * q.inv_tv) * C * exp(-q.env_a * x * x);
    case 1: return C * exp(-q.env_a * x * x);
    case 2: return C / cosh(x * q.inv_tv);
    default: return x > 0.0 ? C : C * exp(-q.env_a * x * x);
  }
}

template <bool kLo, typename T>
__global__ void __launch_bounds__(256) k_seed_tfsf(StencilP<T> p, SeedP q,
                                                   const StepState* __restrict__ st,
                                                   V4<T>* __restrict__ nxt,
                                                   LoV4* __restrict__ nxtlo,
                                                   V4<T>* __restrict__ D) {
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int k = 2 + blockIdx.z;  // 2: scattered-field plane, 3: total-field plane
  if (i > p.nx - 2 || j > p.ny - 2) return;
  const double tn = q.t0 + (double)st->n * q.dt;  // time of level n
  // the incident potential on the other plane of the pair
  const double zo = (k == 2) ? q.z3 : q.z2;
  const double s = seed_signal(q, q.tau_t * tn + q.tau_z * zo + q.tau_c - q.t0o);
  const double sign = (k == 2) ? -1.0 : 1.0;
  const T cx = (T)(sign * (double)p.rz2 * q.ax * s);
  const T cy = (T)(sign * (double)p.rz2 * q.ay * s);
  const V4<T> corr = v4(cx, cy, (T)0, (T)0);
  const long long c = cidx(i, j, k, p.nx, p.nxy);
  D[c] = D[c] + corr;
  if (kLo) {
    V4<T> h, l;
    comp_add(nxt[c], ld_lo<T>(nxtlo, c), corr, &h, &l);
    nxt[c] = h;
    st_lo(nxtlo, c, l);
  } else {
    nxt[c] = nxt[c] + corr;
  }
}

// The Gaussian-beam seed: the incident field varies across the planes, so
// the coupling of vertex (i, j) of one plane to the other is that of the
// NSFD update itself,
//   g(i,j) kz2 + kxA (g(i+1,j) + g(i-1,j) - 2 g(i,j))
//              + kyA (g(i,j+1) + g(i,j-1) - 2 g(i,j)),
// g the incident value on the other plane (x and y neighbour differences on
// planes k +- 1 carry the weights rx^2 A and ry^2 A).  A CTA takes a 16 x 16
// tile of columns and one plane of the pair (blockIdx.z): it evaluates g once
// per vertex of the tile's 18 x 18 halo on the other plane in shared memory,
// then corrects its tile on its own plane.
constexpr int kSeedTile = 16;

// Scalar of the paraxial beam at a rest-frame point: A = (ax, ay) times it.
// Per transverse axis a (xi along p, eta across it), with
// s_a = zeta^2 + z_a^2: amplitude (z_a^2 / s_a)^(1/4), exponent
// -a^2 z_a^2 / (w_a^2 s_a), delay a^2 zeta / (2 c s_a), phase atan(zeta/z_a)/2.
// zeta and tau depend only on the plane's z and the time, so everything but
// the transverse terms is taken once per plane (BeamPlane).
struct BeamPlane {
  double zeta, tau, amp, gouy, ep, eq, isp, isq;
};

__device__ inline BeamPlane beam_plane(const SeedP& q, double z, double t) {
  BeamPlane b;
  b.zeta = q.zeta_t * t + q.zeta_z * z + q.zeta_c;
  b.tau = q.tau_t * t + q.tau_z * z + q.tau_c - q.t0o;
  const double z2 = b.zeta * b.zeta;
  const double sp = z2 + q.zr_p * q.zr_p, sq = z2 + q.zr_q * q.zr_q;
  const double fp = q.zr_p * q.zr_p / sp, fq = q.zr_q * q.zr_q / sq;
  b.amp = sqrt(sqrt(fp * fq));
  b.gouy = 0.5 * (atan2(b.zeta, q.zr_p) + atan2(b.zeta, q.zr_q));
  b.ep = q.inv_w2p * fp;
  b.eq = q.inv_w2q * fq;
  b.isp = 1.0 / sp;
  b.isq = 1.0 / sq;
  return b;
}

__device__ inline double beam_value(const SeedP& q, const BeamPlane& b, double x, double y) {
  const double X = x - q.xf, Y = y - q.yf;
  const double xi = q.px * X + q.py * Y, eta = q.px * Y - q.py * X;
  const double x2 = xi * xi, e2 = eta * eta;
  const double delay = (x2 * b.isp + e2 * b.isq) * b.zeta * (0.5 / kC);
  return b.amp * exp(-(x2 * b.ep + e2 * b.eq)) * seed_signal(q, b.tau - delay, b.gouy);
}

template <bool kLo, typename T>
__global__ void __launch_bounds__(kSeedTile * kSeedTile)
    k_seed_tfsf_beam(StencilP<T> p, SeedP q, const StepState* __restrict__ st,
                     V4<T>* __restrict__ nxt, LoV4* __restrict__ nxtlo,
                     V4<T>* __restrict__ D) {
  constexpr int H = kSeedTile + 2;
  __shared__ double g[H][H];  // the incident scalar on the other plane
  __shared__ BeamPlane bp;
  const int k = 2 + blockIdx.z;  // the corrected plane: 2 scattered, 3 total field
  const int i0 = 1 + blockIdx.x * kSeedTile, j0 = 1 + blockIdx.y * kSeedTile;
  const int tid = threadIdx.y * kSeedTile + threadIdx.x;
  if (tid == 0) {
    const double tn = q.t0 + (double)st->n * q.dt;  // time of level n
    bp = beam_plane(q, k == 2 ? q.z3 : q.z2, tn);
  }
  __syncthreads();
  for (int h = tid; h < H * H; h += kSeedTile * kSeedTile) {
    const int a = h % H, b = h / H;
    const int ii = i0 - 1 + a, jj = j0 - 1 + b;  // >= 0; used only up to nx-1, ny-1
    double v = 0.0;
    if (ii < p.nx && jj < p.ny) v = beam_value(q, bp, q.gx0 + ii * q.gdx, q.gy0 + jj * q.gdy);
    g[b][a] = v;
  }
  __syncthreads();
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  if (i > p.nx - 2 || j > p.ny - 2) return;
  const int a = threadIdx.x + 1, b = threadIdx.y + 1;
  const double c0 = g[b][a];
  const double cpl = c0 * q.kz2 + q.kxA * ((g[b][a + 1] - c0) + (g[b][a - 1] - c0)) +
                     q.kyA * ((g[b + 1][a] - c0) + (g[b - 1][a] - c0));
  const double sgn = (k == 2) ? -1.0 : 1.0;
  const V4<T> corr = v4((T)(sgn * q.ax * cpl), (T)(sgn * q.ay * cpl), (T)0, (T)0);
  const long long c = cidx(i, j, k, p.nx, p.nxy);
  D[c] = D[c] + corr;
  if (kLo) {
    V4<T> hh, ll;
    comp_add(nxt[c], ld_lo<T>(nxtlo, c), corr, &hh, &ll);
    nxt[c] = hh;
    st_lo(nxtlo, c, ll);
  } else {
    nxt[c] = nxt[c] + corr;
  }
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
// The Mur vertices are written by k_mur_boundary before this kernel.
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
    tma_load_field(base, &tm_cur, i0 - 1, j0 - 1, kb - 1 + q, &full[s]);
    if (cols) {
      tma_load_field(base + OFF_D, &tm_d, i0, j0, kd, &full[s]);
      tma_load_field(base + OFF_S, &tm_s, i0, j0, kd, &full[s]);
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
      const long long c = (long long)k * p.nxy + col;
      if (nonzero(sv)) src[c] = zero;
      if (!p.space_charge) dp.w = (T)0;
      D[c] = dp;
      nxt[c] = c0 + dp;
    }
    cm = c0; Xm = X0; Ym = Y0;
    c0 = cp; X0 = Xp; Y0 = Yp;
  }
}

// E and B at vertex v (interior) at t = (n+1/2) dt from psi^{n+1} (pn) and
// the increment D = psi^{n+1} - psi^n:  B = (curl A^n + curl A^{n+1}) / 2 is
// the curl of the mid level pn - D/2; E = -D_A / dt - grad phi^n with
// phi^n = pn.w - D.w; central differences.
// Central differences of the level psi^{n+1} + lo and of D between the
// neighbours a+ and a- of a vertex, A at the mid level (psi^{n+1} - D/2)
// and phi at level n (psi^{n+1} - D): the parts are differenced apart
// (neighbouring hi values subtract exactly), so that the lo parts of the
// compensated forms reach E and B.
template <typename T>
__device__ inline V4<T> level_diff(V4<T> hp, V4<T> hm, V4<T> dp, V4<T> dm) {
  const T half = (T)0.5;
  return v4((hp.x - hm.x) - half * (dp.x - dm.x), (hp.y - hm.y) - half * (dp.y - dm.y),
            (hp.z - hm.z) - half * (dp.z - dm.z), (hp.w - hm.w) - (dp.w - dm.w));
}

// E and B at t = (n+1/2) dt (Sec. "Field Evaluation") from the differences
// along x, y, z (level_diff) and the increment dc at the vertex.
template <typename T>
__device__ inline void eb_from_diffs(const PicP<T>& p, V4<T> gx, V4<T> gy, V4<T> gz, V4<T> dc,
                                     T E[3], T B[3]) {
  B[0] = gy.z * p.inv2dy - gz.y * p.inv2dz;
  B[1] = gz.x * p.inv2dz - gx.z * p.inv2dx;
  B[2] = gx.y * p.inv2dx - gy.x * p.inv2dy;
  E[0] = -dc.x * p.invdt - gx.w * p.inv2dx;
  E[1] = -dc.y * p.invdt - gy.w * p.inv2dy;
  E[2] = -dc.z * p.invdt - gz.w * p.inv2dz;
}

// Adds the lo-part differences around global vertex v (p.plo set).
template <typename T>
__device__ inline void add_lo_diffs(const PicP<T>& p, long long v, V4<T>& gx, V4<T>& gy,
                                    V4<T>& gz) {
  const LoV4* lo = p.plo;
  gx = gx + (ld_lo<T>(lo, v + 1) - ld_lo<T>(lo, v - 1));
  gy = gy + (ld_lo<T>(lo, v + p.nx) - ld_lo<T>(lo, v - p.nx));
  gz = gz + (ld_lo<T>(lo, v + p.nxy) - ld_lo<T>(lo, v - p.nxy));
}

// E and B at interior vertex v from the level pn = psi^{n+1} (lo parts in
// p.plo; kLo = false: the caller knows there are none) and the increment
// D = psi^{n+1} - psi^n.
template <bool kLo = true, typename T>
__device__ inline void eb_vertex(const PicP<T>& p, const V4<T>* __restrict__ pn,
                                 const V4<T>* __restrict__ D, long long v, T E[3], T B[3]) {
  const long long nxy = p.nxy;
  const int nx = p.nx;
  V4<T> gx = level_diff(ldg4(pn + v + 1), ldg4(pn + v - 1), ldg4(D + v + 1), ldg4(D + v - 1));
  V4<T> gy = level_diff(ldg4(pn + v + nx), ldg4(pn + v - nx), ldg4(D + v + nx), ldg4(D + v - nx));
  V4<T> gz =
      level_diff(ldg4(pn + v + nxy), ldg4(pn + v - nxy), ldg4(D + v + nxy), ldg4(D + v - nxy));
  if (kLo && p.plo) add_lo_diffs(p, v, gx, gy, gz);
  eb_from_diffs(p, gx, gy, gz, ldg4(D + v), E, B);
}

__device__ inline bool interior(int i, int j, int k, int nx, int ny, int nz) {
  return i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
}

// Whole-grid copy-out of one field (double), E/B evaluated on the fly.
// what: 0..2 E, 3..5 B, 6..9 component of lev (A_x, A_y, A_z, phi), 10..13
// component of src.
template <typename T>
__global__ void k_extract(PicP<T> p, const V4<T>* __restrict__ pn, const V4<T>* __restrict__ D,
                          const V4<T>* __restrict__ lev, const LoV4* __restrict__ levlo,
                          const V4<T>* __restrict__ src, int what, double* __restrict__ out) {
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
      if (what < 10 && levlo) {
        const V4<T> l = ld_lo<T>(levlo, c);
        val += (double)(comp == 0 ? l.x : comp == 1 ? l.y : comp == 2 ? l.z : l.w);
      }
    }
    out[c] = val;
  }
}

// Host field -> one component of a device array.
template <typename T>
__global__ void k_insert(long long ncell, const double* __restrict__ in, V4<T>* __restrict__ dst,
                         LoV4* __restrict__ dstlo, int comp) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const T v = (T)in[c];
    V4<T> a = dst[c];
    if (comp == 0) a.x = v; else if (comp == 1) a.y = v; else if (comp == 2) a.z = v; else a.w = v;
    dst[c] = a;
    if (dstlo) {  // the rest of the double value below hi
      const T r = (T)(in[c] - (double)v);
      V4<T> l = ld_lo<T>(dstlo, c);
      if (comp == 0) l.x = r; else if (comp == 1) l.y = r; else if (comp == 2) l.z = r; else l.w = r;
      st_lo(dstlo, c, l);
    }
  }
}

// D = newest - previous level (after a level was set from the host).
template <typename T>
__global__ void k_increment(long long ncell, const V4<T>* __restrict__ pn,
                            const V4<T>* __restrict__ po, const LoV4* __restrict__ pnlo,
                            const LoV4* __restrict__ polo, V4<T>* __restrict__ D) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x)
    D[c] = pnlo ? (pn[c] - po[c]) + (ld_lo<T>(pnlo, c) - ld_lo<T>(polo, c)) : pn[c] - po[c];
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
// P = sum (E'_x B'_y - E'_y B'_x) / mu0 dx dy over interior (i, j), the
// part of block bidx of nblocks.
template <typename T>
__device__ __forceinline__ void power_body(const PicP<T>& p, const V4<T>* __restrict__ pn,
                                           const V4<T>* __restrict__ D, int kp, double g0,
                                           double b0, double* __restrict__ acc,
                                           const StepState* __restrict__ st, long long cap,
                                           int slot_from_state, int* __restrict__ err, int bidx,
                                           int nblocks) {
  long long slot = 0;
  if (slot_from_state) {
    slot = st->n;
    if (slot >= cap) return;
  }
  const int nin = (p.nx - 2) * (p.ny - 2);
  const double b0c = b0 / kC;  // one FP64 division per thread, not two per vertex
  double part = 0.0;
  for (int t = bidx * blockDim.x + threadIdx.x; t < nin; t += nblocks * blockDim.x) {
    const int i = 1 + t % (p.nx - 2);
    const int j = 1 + t / (p.nx - 2);
    T E[3], B[3];
    eb_vertex(p, pn, D, cidx(i, j, kp, p.nx, p.nxy), E, B);
    const double Ex = E[0], Ey = E[1], Bx = B[0], By = B[1];
    const double exl = g0 * (Ex + b0 * kC * By);
    const double eyl = g0 * (Ey - b0 * kC * Bx);
    const double bxl = g0 * (Bx - b0c * Ey);
    const double byl = g0 * (By + b0c * Ex);
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

// The result is added to *acc (zeroed by the caller); slot_from_state makes
// the kernel write into acc[state->n] (per-step recording) when below cap.
template <typename T>
__global__ void __launch_bounds__(256) k_power(PicP<T> p, const V4<T>* __restrict__ pn,
                                               const V4<T>* __restrict__ D, int kp, double g0,
                                               double b0, double* __restrict__ acc,
                                               const StepState* __restrict__ st, long long cap,
                                               int slot_from_state, int* __restrict__ err) {
  power_body(p, pn, D, kp, g0, b0, acc, st, cap, slot_from_state, err, blockIdx.x, gridDim.x);
}

}  // namespace mithra
