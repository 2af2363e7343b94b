// common.cuh -- shared device definitions of the GB300 FDTD/PIC step.
//
// Storage (both precisions T = float / double):
//   potentials: two ping-pong levels, each nx*ny*nz cells of
//               V4<T> {A_x, A_y, A_z, phi}, cell (i,j,k) at (k*ny + j)*nx + i
//               (x fastest), and the increment D = newest - previous level;
//   sources:    one array of V4<T> {J_x, J_y, J_z, rho};
//   particles:  structure of arrays, double-buffered for the re-sort:
//               int32 cell (linear cell index, -1 once lost), T fraction of
//               the cell along x, y, z in [0, 1), U momentum u = gamma*beta
//               (U = T, or double with FP32 fields), int32 original index.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mithra {

// CODATA 2018 (c and e exact)
constexpr double kC = 299792458.0;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.0 / (kEps0 * kC * kC);
constexpr double kPi = 3.14159265358979323846;

// particles are binned into tiles of kTile^3 cells; a tile is the unit of
// work of the particle kernel
constexpr int kTile = 8;

template <typename T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};

template <typename T>
__host__ __device__ inline V4<T> v4(T x, T y, T z, T w) {
  V4<T> r;
  r.x = x; r.y = y; r.z = z; r.w = w;
  return r;
}
template <typename T>
__host__ __device__ inline V4<T> operator+(V4<T> a, V4<T> b) {
  return v4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
template <typename T>
__host__ __device__ inline V4<T> operator-(V4<T> a, V4<T> b) {
  return v4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
template <typename T>
__host__ __device__ inline V4<T> operator*(T s, V4<T> a) {
  return v4(s * a.x, s * a.y, s * a.z, s * a.w);
}

// Four-component arithmetic of the potential update.  kPack: FP32 as two
// packed pairs (sm_100's paired FP32 add, multiply and fused multiply-add:
// one instruction for two components, each rounded as the scalar operation;
// a - b as fma(b, -1, a), which rounds a - b once); otherwise (and for FP64)
// the component-wise operators.  vfma(s, a, b) is s a + b, vfma4 the same
// with one factor per component.
__device__ inline float2 v4_xy(V4<float> a) { return make_float2(a.x, a.y); }
__device__ inline float2 v4_zw(V4<float> a) { return make_float2(a.z, a.w); }
__device__ inline V4<float> v4_of(float2 xy, float2 zw) { return v4(xy.x, xy.y, zw.x, zw.y); }

template <bool kPack, typename T>
__device__ inline V4<T> vadd(V4<T> a, V4<T> b) {
  if constexpr (kPack && sizeof(T) == 4)
    return v4_of(__fadd2_rn(v4_xy(a), v4_xy(b)), __fadd2_rn(v4_zw(a), v4_zw(b)));
  else
    return a + b;
}
template <bool kPack, typename T>
__device__ inline V4<T> vsub(V4<T> a, V4<T> b) {
  if constexpr (kPack && sizeof(T) == 4) {
    const float2 m = make_float2(-1.0f, -1.0f);
    return v4_of(__ffma2_rn(v4_xy(b), m, v4_xy(a)), __ffma2_rn(v4_zw(b), m, v4_zw(a)));
  } else {
    return a - b;
  }
}
template <bool kPack, typename T>
__device__ inline V4<T> vmul(T s, V4<T> a) {
  if constexpr (kPack && sizeof(T) == 4) {
    const float2 ss = make_float2(s, s);
    return v4_of(__fmul2_rn(ss, v4_xy(a)), __fmul2_rn(ss, v4_zw(a)));
  } else {
    return s * a;
  }
}
template <bool kPack, typename T>
__device__ inline V4<T> vfma(T s, V4<T> a, V4<T> b) {
  if constexpr (kPack && sizeof(T) == 4) {
    const float2 ss = make_float2(s, s);
    return v4_of(__ffma2_rn(ss, v4_xy(a), v4_xy(b)), __ffma2_rn(ss, v4_zw(a), v4_zw(b)));
  } else {
    return s * a + b;
  }
}
template <bool kPack, typename T>
__device__ inline V4<T> vfma4(V4<T> s, V4<T> a, V4<T> b) {
  if constexpr (kPack && sizeof(T) == 4)
    return v4_of(__ffma2_rn(v4_xy(s), v4_xy(a), v4_xy(b)),
                 __ffma2_rn(v4_zw(s), v4_zw(a), v4_zw(b)));
  else
    return v4(s.x * a.x, s.y * a.y, s.z * a.z, s.w * a.w) + b;
}

template <typename T>
__device__ inline V4<T> ldg4(const V4<T>* p) {
  return __ldg(p);
}
template <>
__device__ inline V4<float> ldg4<float>(const V4<float>* p) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return v4(v.x, v.y, v.z, v.w);
}
template <>
__device__ inline V4<double> ldg4<double>(const V4<double>* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return v4(a.x, a.y, b.x, b.y);
}

// Lo part of a compensated potential level: four bfloat16 values (8 bytes per
// vertex).  The lo part is at most half an ulp of the float hi part, so its
// 8-bit significand adds 8 bits to the level's precision; rounding it to
// bfloat16 each step costs 2^-9 of an ulp of hi.
struct alignas(8) LoV4 {
  __nv_bfloat162 xy, zw;
};

template <typename T>
__device__ inline V4<T> ld_lo(const LoV4* __restrict__ a, long long i) {
  const uint2 raw = __ldg(reinterpret_cast<const uint2*>(a + i));
  LoV4 v;
  memcpy(&v, &raw, sizeof(v));
  const float2 xy = __bfloat1622float2(v.xy), zw = __bfloat1622float2(v.zw);
  return v4((T)xy.x, (T)xy.y, (T)zw.x, (T)zw.y);
}

template <typename T>
__device__ inline void st_lo(LoV4* __restrict__ a, long long i, V4<T> v) {
  LoV4 r;
  r.xy = __floats2bfloat162_rn((float)v.x, (float)v.y);
  r.zw = __floats2bfloat162_rn((float)v.z, (float)v.w);
  a[i] = r;
}

// Division of non-negative 32-bit integers by an invariant divisor d >= 2 by
// multiplication (Granlund and Montgomery, "Division by Invariant Integers
// using Multiplication", 1994): with m = floor(2^64 / d) + 1 (exactly 2^64 / d
// for powers of two), n / d = floor(n m / 2^64) for all n < 2^32.
struct FastDiv {
  unsigned long long m;
  int d;
};
inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  f.d = d;
  f.m = ~0ull / (unsigned long long)d + 1ull;
  return f;
}
__device__ inline int fdiv(int n, const FastDiv& f) {
  return (int)__umul64hi((unsigned long long)(unsigned)n, f.m);
}

// Device-side simulation clock and status words (one per simulation).
struct StepState {
  long long n;          // field steps completed
  long long n_lost;     // particles lost so far
  int err;              // bit 0: NaN/Inf in a reduction; bit 1: a bounded wait gave up
  int n_tiles;          // dense tiles listed by the last scan (entries 0 .. n_tiles-1)
  int work;             // next dense entry of the tile list to hand out
  int n_sparse;         // sparse tiles, listed after the dense ones
  int work_sparse;      // next sparse entry to hand out
  // per level parity c: nonzero when sources may sit outside the tiles
  // marked in the parity's flag array (see StencilP::dirty), so that the
  // potential update of parity c reads every vertex's sources
  int src_all[2];
};

// Coefficients of the potential update in increment form (r_l = c dt / d_l,
// A of Eq. NSFDCoefficient, zero for the standard scheme) and the Mur beta0
// indexed by the mask of axes along which the boundary vertex lies outside
// the interior (x = 1, y = 2, z = 4).
template <typename T>
struct StencilP {
  int nx, ny, nz;
  long long nxy;
  T rxA, rxB, ryA, ryB, rz2;  // rx^2 A, rx^2 (1 - 2A), ry^2 A, ry^2 (1 - 2A), rz^2
  T sA, sphi;                 // (c dt)^2 mu0 and (c dt)^2 / eps0
  T mb0[8];
  // second-order Mur on face vertices (mur2 != 0): m2[a][0], m2[a][1] =
  // (c dt / d_t)^2 d_a / (2 (c dt + d_a)) for the face normal to axis a and
  // its tangential axes t in the order (y, z), (x, z), (x, y)
  T m2[3][2];
  int mur2;
  int space_charge;
  // Sources to read: one flag per 8^3-cell particle tile (tile index
  // ((k/8) nty + j/8) ntx + i/8 of vertex (i, j, k)), set by the particle
  // step for the tiles its deposits reached; the sources of an unmarked
  // tile are zero, and the z-marching update skips their loads unless
  // *src_all is set.  nullptr: every vertex's sources are read.
  const unsigned char* dirty;
  const int* src_all;
  int ntx, nty;
};

// Everything the particle and field-evaluation kernels need.
template <typename T>
struct PicP {
  int nx, ny, nz;
  long long nxy;
  double x0, y0, z0, dxd, dyd, dzd;
  T inv2dx, inv2dy, inv2dz, inv4dx, inv4dy, inv4dz, invdt;
  // lo parts of the level that E and B are evaluated from (compensated
  // forms), nullptr otherwise; set at each launch beside that level
  const LoV4* plo;
  // Boris: h = qm dtb / (2c), an = qm dtb / 2, and each as a float pair
  // (hi the nearest float, lo the nearest float to the remainder) for the
  // FP32 forms, whose particle loop then runs no FP64 instruction
  double h, an;
  float h_hi, h_lo, an_hi, an_lo;
  T cx, cy, cz;  // c dt_b / (dx, dy, dz): cells moved per unit beta in a sub-step
  int n_sub;
  double t0, dt, dtb;
  // undulator (lab field transformed to the rest frame)
  int und_on, fringe;
  int und_type;              // 0 static, 1 optical plane wave
  double g0, b0c, zent, L, lam_u, inv_lam_u, ku_d;
  T ku, B0, ex_fac, by_fac;  // E_x = ex_fac B'_y, B_y = by_fac B'_y
  // optical: tau = gamma0 (1 - d beta0) t + gamma0 (beta0 - d) z / c + d z0'/c;
  // rest-frame E = (oex, oey) s'(tau), B = (obx, oby) s'(tau)
  int osig;
  double w0_d, cep, t0o, tau_t, tau_z, tau_c;
  T w0, env_a, inv_tv, oex, oey, obx, oby;
  T dtau_cell;               // gamma0 (beta0 - d) dz / c: tau per cell along z
  T g0dz;                    // gamma0 dz: lab length of one cell along z
  T y0f, dyf;                // y0 and dy in T
  // deposit
  T qV;                      // q / V
  T jx, jy, jz;              // (q/V) d_l / dt: J_l per cell of displacement
  // tiles
  int ntx, nty, ntz, nkeys;
  FastDiv fd_nx, fd_nxy;  // cell index -> (i, j, k)
};

// Momentum stored as a float-float pair (hi + lo, |lo| <= ulp(hi)/2: about
// 2^-46 relative, the storage of an FP64 value in 8 bytes) for the FP32 form
// with compensated momenta: the Boris step runs on it in FP32 arithmetic
// without converting to and from FP64, whose pipe is narrow on GB300.
struct alignas(8) FF2 {
  float hi, lo;
};

// Conversions of a stored momentum U (float, double or FF2) to and from FP64,
// and its leading value in the fraction type T.
__host__ __device__ inline double u_dbl(float u) { return (double)u; }
__host__ __device__ inline double u_dbl(double u) { return u; }
__host__ __device__ inline double u_dbl(FF2 u) { return (double)u.hi + (double)u.lo; }
template <typename U>
__host__ __device__ inline U u_from(double x);
template <>
__host__ __device__ inline float u_from<float>(double x) { return (float)x; }
template <>
__host__ __device__ inline double u_from<double>(double x) { return x; }
template <>
__host__ __device__ inline FF2 u_from<FF2>(double x) {
  FF2 r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
template <typename T>
__host__ __device__ inline T u_lead(float u) { return (T)u; }
template <typename T>
__host__ __device__ inline T u_lead(double u) { return (T)u; }
template <typename T>
__host__ __device__ inline T u_lead(FF2 u) { return (T)u.hi; }

// T: type of the in-cell fractions; U: type of the momenta.
template <typename T, typename U>
struct Parts {
  int* cell;
  T* fx;
  T* fy;
  T* fz;
  U* ux;
  U* uy;
  U* uz;
  int* id;
};

__host__ __device__ inline long long cidx(int i, int j, int k, int nx, long long nxy) {
  return (long long)k * nxy + (long long)j * nx + i;
}

// (i, j, k) of a linear cell index (k * ny + j) * nx + i.
template <typename P>
__device__ inline void decode_cell(const P& p, int cell, int* i, int* j, int* k) {
  *k = fdiv(cell, p.fd_nxy);
  const int r = cell - *k * (int)p.nxy;
  *j = fdiv(r, p.fd_nx);
  *i = r - *j * p.nx;
}

// largest value of T below one: a fraction that rounds up to 1 is clamped so
// that the cell decided in FP64 stays the particle's cell
template <typename T>
__host__ __device__ inline T below_one();
template <>
__host__ __device__ inline float below_one<float>() { return 0.99999994f; }
template <>
__host__ __device__ inline double below_one<double>() { return 0.99999999999999989; }

template <typename T>
__device__ inline T to_frac(double f) {
  T r = (T)f;
  return r >= (T)1 ? below_one<T>() : r;
}

}  // namespace mithra
