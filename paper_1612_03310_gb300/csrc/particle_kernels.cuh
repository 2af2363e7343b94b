// particle_kernels.cuh -- macroparticles: set-up, gather + undulator + Boris
// push (Eq. BorisScheme, Eq. fieldInterpolation, Sec. "Undulator Field"),
// current and charge deposition (Sec. "Current Deposition",
// Eq. currentIntegral), and the binning of particles into cell tiles (tile
// counts, their scan, and the slot map through which the next particle step
// reads the particles in tile order).
#pragma once
#include "common.cuh"
#include "field_kernels.cuh"

namespace mithra {

// --- math in the particle's precision ------------------------------------
__device__ inline void sincos_t(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ inline void sincos_t(double a, double* s, double* c) { sincos(a, s, c); }
// cosh and sinh of the same argument from one expm1: with m = e^a - 1,
// sinh a = m (1 + e^{-a}) / 2 (no cancellation for small a) and
// cosh a = (e^a + e^{-a}) / 2.
__device__ inline void coshsinh_t(float a, float* ch, float* sh) {
  const float m = expm1f(a);
  const float inv = 1.0f / (1.0f + m);
  *ch = 0.5f * ((1.0f + m) + inv);
  *sh = 0.5f * m * (1.0f + inv);
}
__device__ inline void coshsinh_t(double a, double* ch, double* sh) {
  *ch = cosh(a);
  *sh = sinh(a);
}
__device__ inline float exp_t(float a) { return expf(a); }
__device__ inline double exp_t(double a) { return exp(a); }

// Rest-frame undulator field.  The lab position of a rest-frame event (z, t)
// is z' = gamma0 (z + beta0 c t); zeta = z' - z'_ent is the distance past the
// entrance.  The large, moving-window part of zeta is kept in FP64 once per
// reference plane kref and time (UndFrame): its phase reduced modulo lambda_u,
// the entrance and exit thresholds and the fringe arguments there.  A
// particle adds its offset from the reference plane, gamma0 dz ((k - kref) +
// f_z), in its own precision T.
template <typename T>
struct UndFrame {
  T ph0;      // ku zeta_ref reduced to (-pi, pi]; optical: carrier phase w0 x_ref + cep
  T thr_lo;   // offsets below this are before the entrance; optical: x_ref = tau_ref - t0
  T thr_hi;   // offsets above this are past the exit
  T a_lo0;    // ku zeta_ref (fringe argument before the entrance)
  T a_hi0;    // ku (zeta_ref - L) (fringe argument past the exit)
};

template <typename T>
__device__ inline UndFrame<T> und_frame(const PicP<T>& p, int kref, double t) {
  UndFrame<T> fr;
  if (p.und_type == 1) {
    // optical: signal argument x = tau - t0 at the reference plane, and the
    // carrier phase there reduced to (-pi, pi], in FP64
    const double x = p.tau_t * t + p.tau_z * (p.z0 + (double)kref * p.dzd) + p.tau_c - p.t0o;
    const double ph = p.w0_d * x + p.cep;
    fr.ph0 = (T)(ph - 2.0 * kPi * rint(ph * (0.5 / kPi)));
    fr.thr_lo = (T)x;
    fr.thr_hi = fr.a_lo0 = fr.a_hi0 = (T)0;
    return fr;
  }
  const double zeta = p.g0 * (p.z0 + (double)kref * p.dzd + p.b0c * t) - p.zent;
  fr.ph0 = (T)(p.ku_d * (zeta - p.lam_u * rint(zeta * p.inv_lam_u)));
  fr.thr_lo = (T)(-zeta);
  fr.thr_hi = p.L > 0.0 ? (T)(p.L - zeta) : (T)3.0e38;
  fr.a_lo0 = (T)(p.ku_d * zeta);
  fr.a_hi0 = (T)(p.ku_d * (zeta - p.L));
  return fr;
}

// Field at transverse position y and offset zl = (k - kref) + f_z cells from
// the frame's reference plane.
// Derivative s'(x) of the optical undulator's signal (the FIELD section's
// list; see mithra_undulator) at x = x_ref + dx with the carrier phase
// ph = ph_ref + w0 dx.
template <typename T>
__device__ inline T signal_derivative(const PicP<T>& p, T x, T ph) {
  T sn, cs;
  sincos_t(ph, &sn, &cs);
  const T dC = -p.w0 * sn;
  switch (p.osig) {
    case 0: {
      const T G = exp_t(-p.env_a * x * x);
      const T k = (T)(-4.0 * 0.69314718055994531) * p.inv_tv;
      return k * G * (cs + x * dC - (T)2 * p.env_a * x * x * cs);
    }
    case 1: {
      const T G = exp_t(-p.env_a * x * x);
      return G * (dC - (T)2 * p.env_a * x * cs);
    }
    case 2: {
      const T u = x * p.inv_tv;
      T ch, sh;
      coshsinh_t(u, &ch, &sh);
      return (dC - cs * p.inv_tv * (sh / ch)) / ch;
    }
    default: {
      if (x > (T)0) return dC;
      const T G = exp_t(-p.env_a * x * x);
      return G * (dC - (T)2 * p.env_a * x * cs);
    }
  }
}

// kOpt selects the optical undulator at compile time (a separate
// instantiation of the particle kernels), so that the static kernels carry
// none of its registers.
template <bool kOpt, typename T>
__device__ inline void undulator_field(const PicP<T>& p, const UndFrame<T>& fr, T y, T zl,
                                       T E[3], T B[3]) {
  E[0] = E[1] = E[2] = (T)0;
  B[0] = B[1] = B[2] = (T)0;
  if (!p.und_on) return;
  if (kOpt) {
    const T dx = p.dtau_cell * zl;
    const T sp = signal_derivative(p, fr.thr_lo + dx, fr.ph0 + p.w0 * dx);
    E[0] = p.oex * sp;
    E[1] = p.oey * sp;
    B[0] = p.obx * sp;
    B[1] = p.oby * sp;
    return;
  }
  const T zr = p.g0dz * zl;  // lab distance from the reference plane
  T ch, sh;
  coshsinh_t(p.ku * y, &ch, &sh);
  T by, bz;
  const bool before = zr < fr.thr_lo;
  const bool after = zr > fr.thr_hi;
  if (before || after) {
    if (!p.fringe) return;
    const T a = (before ? fr.a_lo0 : fr.a_hi0) + p.ku * zr;
    const T e = exp_t((T)(-0.5) * a * a);
    by = p.B0 * ch * a * e;
    bz = p.B0 * sh * e;
  } else {
    T sn, cs;
    sincos_t(fr.ph0 + p.ku * zr, &sn, &cs);
    by = p.B0 * ch * sn;
    bz = p.B0 * sh * cs;
  }
  E[0] = p.ex_fac * by;
  B[1] = p.by_fac * by;
  B[2] = bz;
}

// Trilinear gather of E, B (Eq. fieldInterpolation, w0 = 1 - f, w1 = f) at a
// particle in cell (i, j, k) with fractions f, evaluating E, B at the eight
// vertices from the potentials.
template <bool kLo = true, typename T>
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
        eb_vertex<kLo>(p, pn, D, cidx(i + I, j + J, k + K, p.nx, p.nxy), e, b);
        const T w = wx[I] * wy[J] * wz[K];
        E[0] += w * e[0]; E[1] += w * e[1]; E[2] += w * e[2];
        B[0] += w * b[0]; B[1] += w * b[1]; B[2] += w * b[2];
      }
}

// Float-float numbers (hi + lo, |lo| <= ulp(hi)/2, ~2^-46 relative) by the
// error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum and the
// FMA product split.  The _rn intrinsics keep the compiler from fusing the
// steps whose rounding the transformations rely on.
struct FF {
  float hi, lo;
};
__device__ inline FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ inline FF ff_fast(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ inline FF ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ inline FF ff_add(FF a, FF b) {
  const FF s = ff_two_sum(a.hi, b.hi);
  return ff_fast(s.hi, s.lo + (a.lo + b.lo));
}
__device__ inline FF ff_sub(FF a, FF b) { return ff_add(a, {-b.hi, -b.lo}); }
__device__ inline FF ff_mul(FF a, FF b) {
  const FF p = ff_prod(a.hi, b.hi);
  return ff_fast(p.hi, p.lo + (a.hi * b.lo + a.lo * b.hi));
}
__device__ inline FF ff_mul(FF a, float b) {
  const FF p = ff_prod(a.hi, b);
  return ff_fast(p.hi, p.lo + a.lo * b);
}

// 1/sqrt(x) for x >= 1 in FP64 by the Newton-Raphson iteration for the
// reciprocal square root, y <- y (3 - x y^2) / 2, from an FP32 seed (rsqrtf):
// the error squares each step, one step reaches ~1e-13, two reach FP64
// rounding (used when T is double).  Gives
// 1/gamma = 1/sqrt(1 + u.u) without an FP64 square root or division.
template <typename T>
__device__ inline double rsqrt_nr(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);  // relative error ~1e-13 after one step
  if (sizeof(T) == 8) y = y * (1.5 - 0.5 * x * y * y);  // FP64 rounding
  return y;
}

// 1/sqrt(x) in the momentum type: FP64 as above; FP32 from the rsqrtf seed
// with one FP32 Newton-Raphson step.
__device__ inline float rsqrt_u(float x) {
  const float y = rsqrtf(x);
  return y * (1.5f - 0.5f * x * y * y);
}
__device__ inline double rsqrt_u(double x) { return rsqrt_nr<double>(x); }

// 1/sqrt(x) for x = hi + lo >= 1 (a float pair) to FP32 rounding on FP32
// instructions only: the seed y0 = rsqrtf(hi) and one Newton-Raphson step
// y = y0 + y0 r / 2, with the residual r = 1 - x y0^2 formed in float-float
// (y0^2 split exactly by an FMA).  r carries ~2^-46, the step leaves ~2^-43
// (the square of the seed's error), and the one rounding of the final FMA
// gives the nearest float but for near-ties -- what the same Newton step in
// FP64 followed by a conversion to float gives, without GB300's narrow FP64
// pipe.
__device__ inline float rsqrt_ff(float hi, float lo) {
  const float y0 = rsqrtf(hi);
  const FF r = ff_sub(FF{1.0f, 0.0f}, ff_mul(FF{hi, lo}, ff_prod(y0, y0)));
  return fmaf(0.5f * y0, r.hi, y0);
}

// 1/gamma = 1/sqrt(1 + u.u) that moves the particle, recomputed from the
// momentum whatever its type, to the rounding of the fraction type T.
// FP64 momenta: 1 + u.u in FP64, rsqrt_nr.  FP32 momenta: 1 + u.u is first
// formed exactly enough in FP32 pairs -- each square split into its rounded
// value and the exact remainder by an FMA, the seven terms summed with
// TwoSum (error ~2^-48) -- then rsqrt_ff (an FP64 T takes the pair to FP64
// and rsqrt_nr instead).
template <typename T>
__device__ inline T inv_gamma(const double u[3]) {
  return (T)rsqrt_nr<T>(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}
template <typename T>
__device__ inline T inv_gamma_pair(float hi, float lo) {
  if constexpr (sizeof(T) == 4) {
    return rsqrt_ff(hi, lo);
  } else {
    return (T)rsqrt_nr<T>((double)hi + (double)lo);
  }
}
template <typename T>
__device__ inline T inv_gamma(const float u[3]) {
  float hi = 1.0f, lo = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // (the _rn intrinsics keep the compiler from fusing these into FMAs)
    const float p = __fmul_rn(u[a], u[a]);
    const float e = fmaf(u[a], u[a], -p);  // u^2 = p + e exactly
    const float s = __fadd_rn(hi, p);      // TwoSum(hi, p)
    const float bp = __fsub_rn(s, hi);
    lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp)) + e;
    hi = s;
  }
  return inv_gamma_pair<T>(hi, lo);
}

// 1/gamma from float-float momenta: 1 + u.u summed in FP32 pairs (each hi^2
// split exactly by an FMA, the cross terms 2 hi lo and the remainders added
// to the low word), then rsqrt_ff as for FP32 momenta.
template <typename T>
__device__ inline T inv_gamma(const FF2 u[3]) {
  float hi = 1.0f, lo = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p = __fmul_rn(u[a].hi, u[a].hi);
    const float e = fmaf(u[a].hi, u[a].hi, -p) + 2.0f * u[a].hi * u[a].lo;
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp)) + e;
    hi = s;
  }
  return inv_gamma_pair<T>(hi, lo);
}

// Boris rotation and kicks (Eq. BorisScheme) for charge-to-mass qm folded
// into h = qm dtb / (2c) and an = qm dtb / 2, in the momentum type U.  The
// gamma of the half-kicked momentum t1, which only sets the rotation angle,
// is taken in U as well; the gamma that moves the particle is recomputed by
// the caller (inv_gamma).
template <typename T, typename U>
__device__ inline void boris(const PicP<T>& p, U u[3], const T Ef[3], const T Bf[3]) {
  U h, an;
  if constexpr (sizeof(U) == 4) {
    h = p.h_hi;
    an = p.an_hi;
  } else {
    h = (U)p.h;
    an = (U)p.an;
  }
  const U E[3] = {(U)Ef[0], (U)Ef[1], (U)Ef[2]};
  const U B[3] = {(U)Bf[0], (U)Bf[1], (U)Bf[2]};
  const U t1x = u[0] + h * E[0], t1y = u[1] + h * E[1], t1z = u[2] + h * E[2];
  const U ig1 = rsqrt_u((U)1 + t1x * t1x + t1y * t1y + t1z * t1z);
  const U al = an * ig1;
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

// Compensated momenta next to FP32 fields (P32_U64): the momenta are stored
// as float-float pairs (FF2) and the Boris step runs in float-float
// arithmetic on FP32 instructions (GB300's FP64 pipe is narrow): kicks,
// gamma_1 by an FP32 seed and one float-float Newton-Raphson step, the
// rotation vectors t and s (2 / (1 + t.t) by a Newton reciprocal) and both
// cross products carry ~2^-46, far below the FP32 fields they act with.
__device__ inline void boris_ff(const PicP<float>& p, FF u[3], const float Ef[3],
                                const float Bf[3]) {
  const FF h{p.h_hi, p.h_lo}, an{p.an_hi, p.an_lo};
  const FF hE[3] = {ff_mul(h, Ef[0]), ff_mul(h, Ef[1]), ff_mul(h, Ef[2])};
  const FF t1[3] = {ff_add(u[0], hE[0]), ff_add(u[1], hE[1]), ff_add(u[2], hE[2])};
  // 1 / gamma_1 = 1 / sqrt(1 + t1.t1)
  const FF g2 = ff_add(ff_add(ff_add(FF{1.0f, 0.0f}, ff_mul(t1[0], t1[0])), ff_mul(t1[1], t1[1])),
                       ff_mul(t1[2], t1[2]));
  const float y0 = rsqrtf(g2.hi);
  const FF e1 = ff_sub(FF{1.0f, 0.0f}, ff_mul(g2, ff_prod(y0, y0)));  // 1 - g2 y0^2, small
  const FF ig1 = ff_two_sum(y0, 0.5f * y0 * e1.hi);
  const FF al = ff_mul(an, ig1);
  const FF t[3] = {ff_mul(al, Bf[0]), ff_mul(al, Bf[1]), ff_mul(al, Bf[2])};
  // f = 2 / (1 + t.t)
  const FF den = ff_add(ff_add(ff_add(FF{1.0f, 0.0f}, ff_mul(t[0], t[0])), ff_mul(t[1], t[1])),
                        ff_mul(t[2], t[2]));
  const float r0 = 1.0f / den.hi;
  const FF e2 = ff_sub(FF{1.0f, 0.0f}, ff_mul(den, r0));  // 1 - den r0, small
  const FF f = ff_two_sum(2.0f * r0, 2.0f * r0 * e2.hi);
  const FF sv[3] = {ff_mul(f, t[0]), ff_mul(f, t[1]), ff_mul(f, t[2])};
  const FF t2[3] = {ff_add(t1[0], ff_sub(ff_mul(t1[1], t[2]), ff_mul(t1[2], t[1]))),
                    ff_add(t1[1], ff_sub(ff_mul(t1[2], t[0]), ff_mul(t1[0], t[2]))),
                    ff_add(t1[2], ff_sub(ff_mul(t1[0], t[1]), ff_mul(t1[1], t[0])))};
  const FF c[3] = {ff_sub(ff_mul(t2[1], sv[2]), ff_mul(t2[2], sv[1])),
                   ff_sub(ff_mul(t2[2], sv[0]), ff_mul(t2[0], sv[2])),
                   ff_sub(ff_mul(t2[0], sv[1]), ff_mul(t2[1], sv[0]))};
  for (int a = 0; a < 3; ++a) u[a] = ff_add(ff_add(t1[a], c[a]), hE[a]);
}

template <>
__device__ inline void boris<float, FF2>(const PicP<float>& p, FF2 u[3], const float Ef[3],
                                         const float Bf[3]) {
  FF v[3] = {{u[0].hi, u[0].lo}, {u[1].hi, u[1].lo}, {u[2].hi, u[2].lo}};
  boris_ff(p, v, Ef, Bf);
  for (int a = 0; a < 3; ++a) {
    u[a].hi = v[a].hi;
    u[a].lo = v[a].lo;
  }
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

// Splits an offset in cells (relative to cell index c0) into the cell index
// and the fraction in [0, 1), in the fraction type T.
template <typename T>
__device__ inline int split_cell_t(int c0, T s, T* frac) {
  const T fl = floor(s);
  T r = s - fl;
  if (r >= (T)1) r = below_one<T>();
  *frac = r;
  return c0 + (int)fl;
}

// n_sub Boris steps of one particle (Eq. BorisScheme) with the grid E, B from
// gather(i, j, k, f, E, B) and the undulator at each sub-step time, through
// the frame frame(m, k, &kref) of sub-step m; 1/gamma by inv_gamma, the position
// advanced in cells (fraction type T, carry into the cell index).  disp
// receives the displacement in cells over the field step.  Returns false when
// the particle leaves the valid cells.
template <bool kOpt, typename T, typename U, typename Gather, typename Frame>
__device__ inline bool push_particle(const PicP<T>& p, int& i, int& j, int& k, T f[3], U u[3],
                                     T disp[3], Gather&& gather, Frame&& frame) {
  disp[0] = disp[1] = disp[2] = (T)0;
  for (int m = 0; m < p.n_sub; ++m) {
    T E[3], B[3], Eu[3], Bu[3];
    gather(i, j, k, f, E, B);
    int kref;
    const UndFrame<T> fr = frame(m, k, &kref);
    const T y = p.y0f + ((T)j + f[1]) * p.dyf;
    undulator_field<kOpt>(p, fr, y, (T)(k - kref) + f[2], Eu, Bu);
    for (int e = 0; e < 3; ++e) { E[e] += Eu[e]; B[e] += Bu[e]; }
    boris(p, u, E, B);
    const T ig = inv_gamma<T>(u);
    const T d[3] = {p.cx * ig * u_lead<T>(u[0]), p.cy * ig * u_lead<T>(u[1]),
                    p.cz * ig * u_lead<T>(u[2])};
    i = split_cell_t(i, f[0] + d[0], &f[0]);
    j = split_cell_t(j, f[1] + d[1], &f[1]);
    k = split_cell_t(k, f[2] + d[2], &f[2]);
    disp[0] += d[0]; disp[1] += d[1]; disp[2] += d[2];
    if (!valid_cell(i, j, k, p.nx, p.ny, p.nz)) return false;
  }
  return true;
}

// Particle at position from of buffer a to position to of buffer b (lost
// particles, which the particle step moves without pushing them).
template <typename T, typename U>
__device__ inline void copy_particle(const Parts<T, U>& a, const Parts<T, U>& b, long long from,
                                     long long to) {
  b.cell[to] = a.cell[from];
  b.fx[to] = a.fx[from];
  b.fy[to] = a.fy[from];
  b.fz[to] = a.fz[from];
  b.ux[to] = a.ux[from];
  b.uy[to] = a.uy[from];
  b.uz[to] = a.uz[from];
  b.id[to] = a.id[from];
}

// One field step of every particle: n_sub Boris steps with the grid E, B at
// t = (n+1/2) dt held fixed and the undulator at each sub-step time, then the
// deposit of J^{n+1} at the mid point of the path and rho^{n+3/2} at the end,
// and the key/rank of the particle's new tile for the re-sort.  Slot q's
// particle is read at position perm[q] of P and written to slot q of O.
template <bool kOpt, typename T, typename U, bool kLo = false>
__global__ void __launch_bounds__(256) k_push(PicP<T> p, const StepState* __restrict__ st,
                                              const V4<T>* __restrict__ pn,
                                              const V4<T>* __restrict__ D,
                                              V4<T>* __restrict__ src, Parts<T, U> P,
                                              Parts<T, U> O, const int* __restrict__ perm,
                                              long long np, int* __restrict__ count,
                                              int* __restrict__ key, int* __restrict__ rank,
                                              long long* __restrict__ lost_ctr) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const long long pos = perm[q];
  const int cell = P.cell[pos];
  int kk = p.nkeys;  // bucket of lost particles
  if (cell < 0) copy_particle(P, O, pos, q);
  if (cell >= 0) {
    O.id[q] = P.id[pos];
    int i, j, k;
    decode_cell(p, cell, &i, &j, &k);
    T f[3] = {P.fx[pos], P.fy[pos], P.fz[pos]};
    U u[3] = {P.ux[pos], P.uy[pos], P.uz[pos]};
    const int i0 = i, j0 = j, k0 = k;
    const T f0[3] = {f[0], f[1], f[2]};
    T disp[3];
    const double th = p.t0 + ((double)st->n + 0.5) * p.dt;
    const bool ok = push_particle<kOpt>(
        p, i, j, k, f, u, disp,
        [&](int a, int b, int c, const T* ff, T* E, T* B) {
          gather_eb<kLo>(p, pn, D, a, b, c, ff[0], ff[1], ff[2], E, B);
        },
        [&](int m, int kc, int* kref) {
          *kref = kc;
          return und_frame(p, kc, th + m * p.dtb);
        });
    O.ux[q] = u[0]; O.uy[q] = u[1]; O.uz[q] = u[2];
    if (!ok) {
      O.cell[q] = -1;
      O.fx[q] = f0[0]; O.fy[q] = f0[1]; O.fz[q] = f0[2];
      atomicAdd(reinterpret_cast<unsigned long long*>(lost_ctr), 1ULL);
    } else {
      O.cell[q] = (int)cidx(i, j, k, p.nx, p.nxy);
      O.fx[q] = f[0]; O.fy[q] = f[1]; O.fz[q] = f[2];
      // rho^{n+3/2} at the end position
      deposit_cic(p, src, i, j, k, f[0], f[1], f[2], (T)0, (T)0, (T)0, p.qV);
      // J^{n+1} at the mid point of the path
      T mf[3];
      const int mi = split_cell_t(i0, f0[0] + (T)0.5 * disp[0], &mf[0]);
      const int mj = split_cell_t(j0, f0[1] + (T)0.5 * disp[1], &mf[1]);
      const int mk = split_cell_t(k0, f0[2] + (T)0.5 * disp[2], &mf[2]);
      deposit_cic(p, src, mi, mj, mk, mf[0], mf[1], mf[2], p.jx * disp[0], p.jy * disp[1],
                  p.jz * disp[2], (T)0);
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
  P.ux[q] = u_from<U>(ux[q]); P.uy[q] = u_from<U>(uy[q]); P.uz[q] = u_from<U>(uz[q]);
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
  int i, j, k;
  decode_cell(p, cell, &i, &j, &k);
  deposit_cic(p, src, i, j, k, P.fx[q], P.fy[q], P.fz[q], (T)0, (T)0, (T)0, p.qV);
}

// Block-wide exclusive scan of one int per thread (blockDim a multiple of 32,
// at most 1024); *total receives the block sum.  Uses ws[32] shared ints.
__device__ inline int block_exclusive_scan(int v, int* ws, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) ws[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    ws[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  *total = ws[31];
  return incl - v + (wid > 0 ? ws[wid - 1] : 0);
}

// Exclusive scan of the per-tile counts in two coalesced passes over blocks of
// kScanBlock entries.  Pass 1 writes each block's sums (particles, dense
// tiles, sparse tiles).  Pass 2 scans those sums, then its block: offset[t]
// (offset[nkeys+1] = total), the list of non-empty tiles (key < nkeys; key
// nkeys holds the lost particles) for the tiled particle kernel -- tiles with
// at least sparse_below particles first (dense), then the others (sparse),
// each group in key order -- the reset counts, and, in block 0, the two tile
// counts, the reset work counters and (advance != 0: the last kernel of a
// step) the step counter.  sparse_below = 0 lists every tile as dense.
constexpr int kScanBlock = 1024;

__device__ inline void tile_class(int c, int t, int nkeys, int sparse_below, int* dense,
                                  int* sparse) {
  const bool nonempty = c > 0 && t < nkeys;
  *dense = (nonempty && c >= sparse_below) ? 1 : 0;
  *sparse = (nonempty && c < sparse_below) ? 1 : 0;
}

__device__ __forceinline__ void scan_partials_body(const int* __restrict__ count, int nkeys,
                                                   int sparse_below, int4* __restrict__ part,
                                                   int bidx) {
  __shared__ int ws[32];
  const int t = bidx * kScanBlock + threadIdx.x;
  const int c = (t <= nkeys) ? count[t] : 0;
  int dn, sp;
  tile_class(c, t, nkeys, sparse_below, &dn, &sp);
  int tot, nd, ns;
  block_exclusive_scan(c, ws, &tot);
  block_exclusive_scan(dn, ws, &nd);
  block_exclusive_scan(sp, ws, &ns);
  if (threadIdx.x == 0) part[bidx] = make_int4(tot, nd, ns, 0);
}

__global__ void __launch_bounds__(kScanBlock) k_scan_partials(const int* __restrict__ count,
                                                              int nkeys, int sparse_below,
                                                              int4* __restrict__ part) {
  scan_partials_body(count, nkeys, sparse_below, part, blockIdx.x);
}

__device__ __forceinline__ void scan_final_body(int* __restrict__ count, int* __restrict__ offset,
                                                int* __restrict__ tiles, int nkeys,
                                                int sparse_below, const int4* __restrict__ part,
                                                int nblocks, StepState* __restrict__ st,
                                                int advance, int bidx) {
  __shared__ int ws[32];
  __shared__ int base[3], total[3];
  // bases of this block from the block sums (nblocks <= kScanBlock)
  const int4 pv = (threadIdx.x < nblocks) ? part[threadIdx.x] : make_int4(0, 0, 0, 0);
  int all_c, all_d, all_s;
  const int bc = block_exclusive_scan(pv.x, ws, &all_c);
  const int bd = block_exclusive_scan(pv.y, ws, &all_d);
  const int bs = block_exclusive_scan(pv.z, ws, &all_s);
  if (threadIdx.x == bidx) { base[0] = bc; base[1] = bd; base[2] = bs; }
  if (threadIdx.x == 0) { total[0] = all_c; total[1] = all_d; total[2] = all_s; }
  __syncthreads();
  const int t = bidx * kScanBlock + threadIdx.x;
  const int c = (t <= nkeys) ? count[t] : 0;
  int dn, sp;
  tile_class(c, t, nkeys, sparse_below, &dn, &sp);
  int dummy;
  const int off = base[0] + block_exclusive_scan(c, ws, &dummy);
  const int sd = base[1] + block_exclusive_scan(dn, ws, &dummy);
  const int ss = total[1] + base[2] + block_exclusive_scan(sp, ws, &dummy);
  if (t <= nkeys) {
    offset[t] = off;
    count[t] = 0;
    if (dn) tiles[sd] = t;
    if (sp) tiles[ss] = t;
  }
  if (bidx == 0 && threadIdx.x == 0) {
    offset[nkeys + 1] = total[0];
    st->n_tiles = total[1];
    st->n_sparse = total[2];
    st->work = 0;
    st->work_sparse = 0;
    if (advance) st->n += 1;
  }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_final(int* __restrict__ count,
                                                           int* __restrict__ offset,
                                                           int* __restrict__ tiles, int nkeys,
                                                           int sparse_below,
                                                           const int4* __restrict__ part,
                                                           int nblocks, StepState* __restrict__ st,
                                                           int advance) {
  scan_final_body(count, offset, tiles, nkeys, sparse_below, part, nblocks, st, advance,
                  blockIdx.x);
}

// The re-sort: slot offset[key] + rank of the next step's tile order gets
// the position q at which the particle step left the particle (the
// particles stay where they are; the next particle step reads each slot's
// particle through this map and writes it to that slot of the other
// buffer).
__device__ __forceinline__ void slot_one(long long q, const int* __restrict__ key,
                                         const int* __restrict__ rank,
                                         const int* __restrict__ offset, int* __restrict__ perm) {
  perm[(long long)offset[key[q]] + rank[q]] = (int)q;
}

// The initial sort: every particle moved to its slot offset[key] + rank of
// the other buffer, and the slot map the identity (the first particle step
// then reads each tile's particles contiguously).
template <typename T, typename U>
__global__ void __launch_bounds__(256) k_sort_particles(Parts<T, U> a, Parts<T, U> b, long long np,
                                                        const int* __restrict__ key,
                                                        const int* __restrict__ rank,
                                                        const int* __restrict__ offset,
                                                        int* __restrict__ perm) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const long long d = (long long)offset[key[q]] + rank[q];
  copy_particle(a, b, q, d);
  perm[d] = (int)d;
}

// kSlotPer particles a thread (strided by the block, so that the loads of
// key and rank stay coalesced), all their loads in flight before the stores.
constexpr int kSlotPer = 4;

__global__ void __launch_bounds__(256) k_slot_map(long long np, const int* __restrict__ key,
                                                  const int* __restrict__ rank,
                                                  const int* __restrict__ offset,
                                                  int* __restrict__ perm) {
  const long long q0 = blockIdx.x * (long long)(blockDim.x * kSlotPer) + threadIdx.x;
  int kk[kSlotPer], rr[kSlotPer];
#pragma unroll
  for (int u = 0; u < kSlotPer; ++u) {
    const long long q = q0 + (long long)u * blockDim.x;
    if (q < np) {
      kk[u] = key[q];
      rr[u] = rank[q];
    }
  }
#pragma unroll
  for (int u = 0; u < kSlotPer; ++u) {
    const long long q = q0 + (long long)u * blockDim.x;
    if (q < np) perm[(long long)offset[kk[u]] + rr[u]] = (int)q;
  }
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
    int i, j, k;
  decode_cell(p, cell, &i, &j, &k);
    x = p.x0 + ((double)i + (double)P.fx[q]) * p.dxd;
    y = p.y0 + ((double)j + (double)P.fy[q]) * p.dyd;
    z = p.z0 + ((double)k + (double)P.fz[q]) * p.dzd;
    lost = 0.0;
  }
  out[0 * np + d] = x;
  out[1 * np + d] = y;
  out[2 * np + d] = z;
  out[3 * np + d] = u_dbl(P.ux[q]);
  out[4 * np + d] = u_dbl(P.uy[q]);
  out[5 * np + d] = u_dbl(P.uz[q]);
  out[6 * np + d] = lost;
}

}  // namespace mithra
