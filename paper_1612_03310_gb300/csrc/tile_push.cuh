// tile_push.cuh -- particle step by cell tiles.
//
// A persistent CTA takes dense 8^3-cell tiles from the list the last re-sort
// produced.  For each tile it
//   1. loads psi^{n+1} and the increment D over the vertices
//      [t0 - 1, t0 + 9]^3 (11^3, two TMA box loads, one mbarrier);
//   2. evaluates E and B at t = (n+1/2) dt at the tile's 9^3 vertices
//      (Sec. "Field Evaluation") into shared memory;
//   3. pushes the tile's particles, each slot's particle read at the
//      position the re-sort's slot map gives and written to the same slot
//      of the other buffer: trilinear gather from shared memory
//      (Eq. fieldInterpolation), rest-frame undulator field, Boris
//      (Eq. BorisScheme; 1/gamma to the particle precision's rounding, by a
//      float-float Newton step in the FP32 forms), cell carry;
//   4. deposits rho^{n+3/2} (end point) into a shared-memory block over the
//      11^3 vertices -- in the FP32 forms as exact int32 fixed-point sums,
//      added to the global sources once per touched vertex -- and
//      J^{n+1} (mid point) with FP32 vector atomics straight into L2 (FP64:
//      both components through a shared FP64 block).
// A particle whose sub-step leaves the tile (n_sub > 1) gathers from global
// memory, and one whose deposit leaves the 11^3 block deposits with global
// atomics: the same arithmetic on another path.  Sparse tiles (fewer
// particles than the staging pays for) are then taken one per warp on that
// global path.  Particles lost in earlier steps are only moved to the
// other buffer and keep their re-sort bucket.
#pragma once
#include "common.cuh"
#include "field_kernels.cuh"
#include "particle_kernels.cuh"
#include "batch_table.cuh"
#include "tma.cuh"

namespace mithra {

constexpr int kTP = kTile + 3;             // potential / deposit vertices per axis
constexpr int kTE = kTile + 1;             // E/B vertices per axis
constexpr int kTPC = kTP * kTP * kTP;      // 1331
constexpr int kTEC = kTE * kTE * kTE;      // 729
constexpr int kPushThreads = 256;          // threads of a particle-step CTA

template <typename T>
__host__ __device__ constexpr int tile_box_bytes() {
  return kTPC * (int)sizeof(V4<T>);
}
template <typename T>
__host__ __device__ constexpr int tile_box_stride() {
  return (tile_box_bytes<T>() + 127) / 128 * 128;
}
template <typename T>
__host__ __device__ constexpr int tile_eb_offset() {
  return 2 * tile_box_stride<T>();
}
// E and B per vertex as (E_x, E_y, E_z, B_x) and (B_y, B_z): 24 instead of
// 32 bytes a vertex in FP32, which keeps three CTAs per SM within the
// 196 KB shared-memory configuration and leaves 60 KB of the SM's L1 to
// register spills and the particles' loads.
template <typename T>
struct alignas(2 * sizeof(T)) V2 {
  T x, y;
};
template <typename T>
__host__ __device__ constexpr int tile_b2_offset() {
  return tile_eb_offset<T>() + kTEC * (int)sizeof(V4<T>);
}
template <typename T>
__host__ __device__ constexpr int tile_bar_offset() {
  return tile_b2_offset<T>() + kTEC * (int)sizeof(V2<T>);
}
template <typename T, typename U>
__host__ __device__ constexpr int tile_smem_bytes() {
  return tile_bar_offset<T>() + 16;
}
// The next-particle slots of the dense loop (one particle per thread: cell,
// fractions, momenta, original index, and the position of the particle
// after it) in the increment box, which is free once E and B are built.
template <typename T>
__host__ __device__ constexpr int tile_slot_offset() {
  return tile_box_stride<T>();
}
template <typename T, typename U>
__host__ __device__ constexpr int tile_slot_bytes() {
  return kPushThreads * (4 + 3 * (int)sizeof(T) + 3 * (int)sizeof(U) + 8);
}

// E, B at local vertex l of the potential box (strides 1, 11, 121), global
// index g (for the lo parts), same arithmetic as eb_vertex.
template <bool kLo, typename T>
__device__ inline void eb_local(const PicP<T>& p, const V4<T>* __restrict__ sP,
                                const V4<T>* __restrict__ sD, int l, long long g, V4<T>& E,
                                V4<T>& B) {
  constexpr int SX = 1, SY = kTP, SZ = kTP * kTP;
  V4<T> gx = level_diff(sP[l + SX], sP[l - SX], sD[l + SX], sD[l - SX]);
  V4<T> gy = level_diff(sP[l + SY], sP[l - SY], sD[l + SY], sD[l - SY]);
  V4<T> gz = level_diff(sP[l + SZ], sP[l - SZ], sD[l + SZ], sD[l - SZ]);
  if (kLo && p.plo) add_lo_diffs(p, g, gx, gy, gz);
  T e[3], b[3];
  eb_from_diffs(p, gx, gy, gz, sD[l], e, b);
  E = v4(e[0], e[1], e[2], (T)0);
  B = v4(b[0], b[1], b[2], (T)0);
}

// CIC deposit into the shared 11^3 block whose vertex (0,0,0) is global
// (i0-1, j0-1, k0-1), one array per component (stride kTPC: J_x, J_y, J_z,
// rho); kRho selects the charge (one component) or the current (three).
// Falls back to global atomics outside the block.
template <bool kRho, typename T>
__device__ inline void deposit_tile(const PicP<T>& p, T* __restrict__ sJ,
                                    V4<T>* __restrict__ src, int i0, int j0, int k0, int i, int j,
                                    int k, T fx, T fy, T fz, T jx, T jy, T jz, T rho) {
  const int li = i - (i0 - 1), lj = j - (j0 - 1), lk = k - (k0 - 1);
  if (li < 0 || li > kTP - 2 || lj < 0 || lj > kTP - 2 || lk < 0 || lk > kTP - 2) {
    deposit_cic(p, src, i, j, k, fx, fy, fz, jx, jy, jz, rho);
    return;
  }
  const T wx[2] = {(T)1 - fx, fx}, wy[2] = {(T)1 - fy, fy}, wz[2] = {(T)1 - fz, fz};
#pragma unroll
  for (int K = 0; K < 2; ++K)
#pragma unroll
    for (int J = 0; J < 2; ++J)
#pragma unroll
      for (int I = 0; I < 2; ++I) {
        const T w = wx[I] * wy[J] * wz[K];
        T* a = sJ + ((lk + K) * kTP + (lj + J)) * kTP + (li + I);
        if (kRho) {
          atomicAdd(a + 3 * kTPC, w * rho);
        } else {
          atomicAdd(a, w * jx);
          atomicAdd(a + kTPC, w * jy);
          atomicAdd(a + 2 * kTPC, w * jz);
        }
      }
}

// Charge deposit of the FP32 forms into the 11^3 block.  Every rho
// contribution is w q/V with a CIC weight w in [0, 1], so the block sums the
// integers hi = rint(w 2^b) and lo = rint((w 2^b - hi) 2^b) with int32
// shared atomics (native, unlike FP32 shared atomics), b = min(21, 30 -
// ceil(log2 n_t)) for the tile's n_t particles: neither sum can overflow
// (n_t 2^b <= 2^30), one contribution is resolved to 2^-2b q/V, and the sums
// do not depend on the order of the atomics.  Rounding to an integer by
// adding 1.5 2^23, exact for |x| < 2^22 (w 2^b <= 2^21; the products by
// powers of two are exact).
__device__ inline void rho_fixed_add(int* __restrict__ hi, int* __restrict__ lo, int v, float w,
                                     float sb) {
  const float M = 12582912.0f;
  const float X = w * sb;
  const float t = X + M;
  const float Y = (X - (t - M)) * sb;
  atomicAdd(hi + v, __float_as_int(t) - __float_as_int(M));
  atomicAdd(lo + v, __float_as_int(Y + M) - __float_as_int(M));
}

template <typename T>
__device__ inline void deposit_rho_fixed(const PicP<T>& p, int* __restrict__ hi,
                                         int* __restrict__ lo, V4<T>* __restrict__ src, int i0,
                                         int j0, int k0, int i, int j, int k, T fx, T fy, T fz,
                                         float sb) {
  const int li = i - (i0 - 1), lj = j - (j0 - 1), lk = k - (k0 - 1);
  if (sb == 0.0f || li < 0 || li > kTP - 2 || lj < 0 || lj > kTP - 2 || lk < 0 ||
      lk > kTP - 2) {
    deposit_cic(p, src, i, j, k, fx, fy, fz, (T)0, (T)0, (T)0, p.qV);
    return;
  }
  const float wx[2] = {1.0f - (float)fx, (float)fx}, wy[2] = {1.0f - (float)fy, (float)fy},
              wz[2] = {1.0f - (float)fz, (float)fz};
#pragma unroll
  for (int K = 0; K < 2; ++K)
#pragma unroll
    for (int J = 0; J < 2; ++J)
#pragma unroll
      for (int I = 0; I < 2; ++I)
        rho_fixed_add(hi, lo, ((lk + K) * kTP + (lj + J)) * kTP + (li + I),
                      wx[I] * wy[J] * wz[K], sb);
}

// One particle's field step (shared by the staged and the per-warp path):
// push, then the deposits of rho at the end point and J at the mid point
// through dep(kRho, i, j, k, f, jx, jy, jz, rho), and the re-sort bucket.
// The particle in slot q of the tile order comes from ld_cell(), ld_fu(f, u)
// and ld_id() (the state buffer at the slot's position) and goes to slot q
// of the output buffer O, complete (a lost particle too), so that O holds
// every particle in slot order.  next() is called once the state has been
// consumed (after the push, or for a lost particle after its loads), where
// the dense loop starts the copy of the thread's next particle into the
// slot it read.
template <bool kOpt, typename T, typename U, typename Gather, typename Frame, typename Dep,
          typename LdCell, typename LdFU, typename LdId, typename Next>
__device__ inline void tile_particle(const PicP<T>& p, const Parts<T, U>& O, long long q,
                                     int* __restrict__ count, int* __restrict__ key,
                                     int* __restrict__ rank, long long* __restrict__ lost_ctr,
                                     Gather&& gather, Frame&& frame, Dep&& dep, LdCell&& ld_cell,
                                     LdFU&& ld_fu, LdId&& ld_id, Next&& next) {
  const int cell = ld_cell();
  const int id = ld_id();
  T f[3];
  U u[3];
  ld_fu(f, u);
  O.id[q] = id;
  int kk = p.nkeys;
  if (cell < 0) {
    next();
    O.cell[q] = cell;
    O.fx[q] = f[0]; O.fy[q] = f[1]; O.fz[q] = f[2];
    O.ux[q] = u[0]; O.uy[q] = u[1]; O.uz[q] = u[2];
  } else {
    int i, j, k;
    decode_cell(p, cell, &i, &j, &k);
    const int ia = i, ja = j, ka = k;
    const T f0[3] = {f[0], f[1], f[2]};
    T disp[3];
    const bool ok = push_particle<kOpt>(p, i, j, k, f, u, disp, gather, frame);
    next();
    O.ux[q] = u[0]; O.uy[q] = u[1]; O.uz[q] = u[2];
    if (!ok) {
      O.cell[q] = -1;
      O.fx[q] = f0[0]; O.fy[q] = f0[1]; O.fz[q] = f0[2];
      atomicAdd(reinterpret_cast<unsigned long long*>(lost_ctr), 1ULL);
    } else {
      O.cell[q] = (int)cidx(i, j, k, p.nx, p.nxy);
      O.fx[q] = f[0]; O.fy[q] = f[1]; O.fz[q] = f[2];
      // the bucket's rank first: its atomic's round trip overlaps the
      // deposits
      kk = tile_key(p, i, j, k);
      const int r = bin_rank(count, kk);
      dep(true, i, j, k, f, (T)0, (T)0, (T)0, p.qV);
      T mf[3];
      const int mi = split_cell_t(ia, f0[0] + (T)0.5 * disp[0], &mf[0]);
      const int mj = split_cell_t(ja, f0[1] + (T)0.5 * disp[1], &mf[1]);
      const int mk = split_cell_t(ka, f0[2] + (T)0.5 * disp[2], &mf[2]);
      dep(false, mi, mj, mk, mf, p.jx * disp[0], p.jy * disp[1], p.jz * disp[2], (T)0);
      key[q] = kk;
      rank[q] = r;
      return;
    }
  }
  key[q] = kk;
  rank[q] = bin_rank(count, kk);
}

template <typename T>
__device__ inline void tile_origin(const PicP<T>& p, int tile, int* i0, int* j0, int* k0) {
  *i0 = (tile % p.ntx) * kTile;
  *j0 = ((tile / p.ntx) % p.nty) * kTile;
  *k0 = (tile / (p.ntx * p.nty)) * kTile;
}

// Kernel parameters of the tiled particle step, all in param space (read
// where used, like constants, instead of held in registers; the tensor maps
// there too, so that no TMA unit can hold a stale copy of a map rewritten in
// global memory): one simulation's arguments and tensor maps, or those of up
// to kPushGroup batch members, whose non-empty tiles, numbered member after
// member by pref, one counter hands out.
constexpr int kPushGroup = 30;  // 30 x (792 + 256) B (FP64) of the 32 KB parameter space

// Member of tile number w of a batch group: pref[m] <= w < pref[m+1].
__device__ inline int member_of_tile(const int* __restrict__ pref, int M, int w) {
  int lo = 0, hi = M - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T, typename U, bool kBatch>
struct PushParams;

template <typename T, typename U>
struct PushParams<T, U, false> {
  CUtensorMap tm_pn;  // psi^{n+1}, 11^3 boxes
  CUtensorMap tm_d;   // increment, 11^3 boxes
  PushArgs<T, U> args;
};

template <typename T, typename U>
struct PushParams<T, U, true> {
  CUtensorMap box[kPushGroup];    // the members' psi^{n+1}, 11^3 boxes
  CUtensorMap box_d[kPushGroup];  // their increments
  PushArgs<T, U> m[kPushGroup];
  const int* pref;  // pref[0 .. M]: tiles before each member
  int* work;        // tile counter
  int M;
};

template <bool kOpt, typename T, typename U, bool kLo = false, bool kBatch = false>
__global__ void __launch_bounds__(kPushThreads, (sizeof(T) == 4 ? 3 : 1))
    k_push_tiled(const __grid_constant__ PushParams<T, U, kBatch> prm) {
  extern __shared__ __align__(128) unsigned char smem[];
  V4<T>* sP = reinterpret_cast<V4<T>*>(smem);
  V4<T>* sD = reinterpret_cast<V4<T>*>(smem + tile_box_stride<T>());
  V4<T>* sE = reinterpret_cast<V4<T>*>(smem + tile_eb_offset<T>());   // E_x..E_z, B_x
  V2<T>* sB = reinterpret_cast<V2<T>*>(smem + tile_b2_offset<T>());   // B_y, B_z
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + tile_bar_offset<T>());
  static_assert(tile_slot_bytes<T, U>() <= tile_box_bytes<T>(), "slots fit the increment box");
  // deposit block, reuses the psi box once E, B are built.  FP64: one array
  // per component (J_x, J_y, J_z, rho), so that atomics of a component from
  // different vertices spread over all banks.  FP32: the fixed-point rho
  // sums (hi, lo), the current going to global memory directly (vector
  // atomics in L2, measured faster than FP32 shared-memory atomics).
  constexpr bool kF32 = sizeof(T) == 4;
  // this thread's next-particle slot (stride kPushThreads between the
  // components), in
  // the increment box: written only after E and B are built, and drained
  // before the CTA's next tile loads into the box
  int* sl_cell = reinterpret_cast<int*>(smem + tile_slot_offset<T>()) + threadIdx.x;
  T* sl_f = reinterpret_cast<T*>(smem + tile_slot_offset<T>() + kPushThreads * 4) + threadIdx.x;
  U* sl_u = reinterpret_cast<U*>(smem + tile_slot_offset<T>() +
                                 kPushThreads * (4 + 3 * (int)sizeof(T))) +
            threadIdx.x;
  int* sl_id = reinterpret_cast<int*>(smem + tile_slot_offset<T>() +
                                      kPushThreads * (4 + 3 * (int)sizeof(T) +
                                                      3 * (int)sizeof(U))) +
               threadIdx.x;
  int* sl_pos = sl_id + kPushThreads;
  T* sJ = reinterpret_cast<T*>(sP);
  int* sRh = reinterpret_cast<int*>(sP);
  int* sRl = sRh + kTPC;
  __shared__ int s_tile;
  constexpr int kMaxFrames = 16;
  __shared__ UndFrame<T> s_frame[kMaxFrames];  // undulator frames of the tile
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  // launched as a programmatic dependent of the potential update (one
  // simulation): the CTAs are placed while the update drains, and wait here,
  // before any global access, for it to complete (a no-op otherwise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  uint32_t phase = 0;
  // Source-tile flags (StencilP::dirty): the array this step's potential
  // update read is cleared, and the deposits mark the other -- a tile's 27
  // neighbours, which hold every vertex a particle of the tile deposits to
  // while its end and mid-point cells stay within [t0 - 8, t0 + 14] on each
  // axis (t0 the tile's first cell); a deposit beyond that sets src_all of
  // the next parity instead.
  auto clear_flags = [&](const PushArgs<T, U>& a) {
    unsigned* f = reinterpret_cast<unsigned*>(a.dirty) + (size_t)a.cur * a.dirty_words;
    for (int w = blockIdx.x * blockDim.x + tid; w < a.dirty_words; w += gridDim.x * blockDim.x)
      f[w] = 0u;
    if (blockIdx.x == 0 && tid == 0) a.st->src_all[a.cur] = 0;
  };
  auto mark_tile = [&](const PushArgs<T, U>& a, int tile, int r) {  // neighbour r of 27
    const PicP<T>& p = a.p;
    const int tx = tile % p.ntx + r % 3 - 1, ty = (tile / p.ntx) % p.nty + (r / 3) % 3 - 1,
              tz = tile / (p.ntx * p.nty) + r / 9 - 1;
    if (tx >= 0 && tx < p.ntx && ty >= 0 && ty < p.nty && tz >= 0 && tz < p.ntz)
      a.dirty[(size_t)(1 - a.cur) * 4 * a.dirty_words + ((size_t)tz * p.nty + ty) * p.ntx + tx] =
          1;
  };
  auto far_deposit = [&](const PushArgs<T, U>& a, int i0, int j0, int k0, int i, int j, int k) {
    if ((unsigned)(i - i0 + 8) > 22u || (unsigned)(j - j0 + 8) > 22u ||
        (unsigned)(k - k0 + 8) > 22u)
      a.st->src_all[1 - a.cur] = 1;
  };
  // the particle at position pos of the state buffer into this thread's
  // slot, and the position of the slot after it (qn, when below end) into
  // sl_pos: issued after the particle's copies, which read the old sl_pos
  auto prefetch = [&](const Parts<T, U>& P, const int* perm, long long pos, long long qn,
                      int end) {
    cp_async<4>(sl_cell, P.cell + pos);
    cp_async<sizeof(T)>(sl_f, P.fx + pos);
    cp_async<sizeof(T)>(sl_f + kPushThreads, P.fy + pos);
    cp_async<sizeof(T)>(sl_f + 2 * kPushThreads, P.fz + pos);
    cp_async<sizeof(U)>(sl_u, P.ux + pos);
    cp_async<sizeof(U)>(sl_u + kPushThreads, P.uy + pos);
    cp_async<sizeof(U)>(sl_u + 2 * kPushThreads, P.uz + pos);
    cp_async<4>(sl_id, P.id + pos);
    if (qn < end) cp_async<4>(sl_pos, perm + qn);
    cp_async_commit();
  };
  // the slots after the last tile's (particles lost before this step): moved
  // to the output buffer, their bucket kept
  auto lost_tail = [&](const PushArgs<T, U>& a) {
    const int nk = a.p.nkeys;
    for (long long q = a.offset[nk] + (long long)blockIdx.x * blockDim.x + tid; q < a.np;
         q += (long long)gridDim.x * blockDim.x) {
      copy_particle(a.P, a.O, a.perm[q], q);
      a.key[q] = nk;
      a.rank[q] = bin_rank(a.count, nk);
    }
  };
  // the dense tiles of one simulation's list, then its sparse tiles and lost
  // tail (each written once; one simulation runs them straight through, a
  // batch member by member)
  // one staged tile: entry t of the simulation's tile list
  auto dense = [&](const PushArgs<T, U>& a, const CUtensorMap* tmp, const CUtensorMap* tmd,
                   int t, double th) {
    const PicP<T>& p = a.p;
    StepState* const& st = a.st;
    const V4<T>* const& pn = a.pn;
    const V4<T>* const& D = a.D;
    V4<T>* const& src = a.src;
    const Parts<T, U>& P = a.P;
    const Parts<T, U>& O = a.O;
    const int* const& perm = a.perm;
    const int* const& offset = a.offset;
    const int* const& tiles = a.tiles;
    int* const& count = a.count;
    int* const& key = a.key;
    int* const& rank = a.rank;
    long long* const& lost_ctr = a.lost_ctr;
    {
      const int tile = tiles[t];
      // the tile's particle range, loaded while the boxes are in flight
      const int beg = offset[tile], end = offset[tile + 1];
      int i0, j0, k0;
      tile_origin(p, tile, &i0, &j0, &k0);
      if (tid == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, 2u * tile_box_bytes<T>());
        tma_load_field(sP, tmp, i0 - 1, j0 - 1, k0 - 1, bar);
        tma_load_field(sD, tmd, i0 - 1, j0 - 1, k0 - 1, bar);
      }
      if (tid < 27) mark_tile(a, tile, tid);
      // the lo parts of psi^{n+1}, which the E/B phase reads from global
      // memory (the update that wrote them has since streamed the grid
      // through L2), asked of L2 while the boxes are in flight: the first
      // and last vertex of each of the box's 11 x 11 rows of 88 bytes
      // (clamped to the grid)
      if (kLo && p.plo && tid < 2 * kTP * kTP) {
        const int r = tid >> 1;
        const int ii = min(max(i0 - 1 + (tid & 1) * (kTP - 1), 0), p.nx - 1);
        const int jj = min(max(j0 - 1 + r % kTP, 0), p.ny - 1);
        const int kk = min(max(k0 - 1 + r / kTP, 0), p.nz - 1);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p.plo + cidx(ii, jj, kk, p.nx, p.nxy)));
      }
      // FP64 moving-window bookkeeping once per tile and sub-step
      for (int m = tid; m < p.n_sub && m < kMaxFrames; m += blockDim.x)
        s_frame[m] = und_frame(p, k0, th + m * p.dtb);
      mbar_wait_bounded(bar, phase, &st->err);
      phase ^= 1u;
      // E and B at the tile's vertices
      for (int v = tid; v < kTEC; v += blockDim.x) {
        const int a = v % kTE, b = (v / kTE) % kTE, c = v / (kTE * kTE);
        V4<T> E = v4((T)0, (T)0, (T)0, (T)0), B = E;
        if (interior(i0 + a, j0 + b, k0 + c, p.nx, p.ny, p.nz))
          eb_local<kLo>(p, sP, sD, ((c + 1) * kTP + (b + 1)) * kTP + (a + 1),
                   cidx(i0 + a, j0 + b, k0 + c, p.nx, p.nxy), E, B);
        sE[v] = v4(E.x, E.y, E.z, B.x);
        sB[v] = V2<T>{B.y, B.z};
      }
      __syncthreads();
      if (beg + tid < end) prefetch(P, perm, perm[beg + tid], beg + tid + kPushThreads, end);
      // fixed-point scale 2^b of the FP32 charge block (0: tiles of more
      // than 2^16 particles deposit rho in global memory)
      float sb = 0.0f;
      int bsh = 0;
      if (kF32) {
        const int nt = end - beg;
        bsh = min(21, 30 - (nt > 1 ? 32 - __clz(nt - 1) : 0));
        if (nt <= 65536) sb = __int_as_float((127 + bsh) << 23);
        for (int c = tid; c < 2 * kTPC; c += blockDim.x) sRh[c] = 0;
      } else {
        for (int c = tid; c < 4 * kTPC; c += blockDim.x) sJ[c] = (T)0;
      }
      __syncthreads();

      for (int q = beg + tid; q < end; q += blockDim.x) {
        cp_async_wait_all();
        tile_particle<kOpt>(
            p, O, q, count, key, rank, lost_ctr,
            [&](int ci, int cj, int ck, const T* ff, T* E, T* B) {
              const int a = ci - i0, b = cj - j0, c = ck - k0;
              if (a >= 0 && a < kTile && b >= 0 && b < kTile && c >= 0 && c < kTile) {
                const T wx[2] = {(T)1 - ff[0], ff[0]}, wy[2] = {(T)1 - ff[1], ff[1]},
                        wz[2] = {(T)1 - ff[2], ff[2]};
                E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = (T)0;
  #pragma unroll
                for (int K = 0; K < 2; ++K)
  #pragma unroll
                  for (int J = 0; J < 2; ++J)
  #pragma unroll
                    for (int I = 0; I < 2; ++I) {
                      const int v = ((c + K) * kTE + (b + J)) * kTE + (a + I);
                      const V4<T> e = sE[v];
                      const V2<T> bb = sB[v];
                      const T w = wx[I] * wy[J] * wz[K];
                      E[0] += w * e.x; E[1] += w * e.y; E[2] += w * e.z;
                      B[0] += w * e.w; B[1] += w * bb.x; B[2] += w * bb.y;
                    }
              } else {
                gather_eb<kLo>(p, pn, D, ci, cj, ck, ff[0], ff[1], ff[2], E, B);
              }
            },
            [&](int m, int kc, int* kref) {
              *kref = k0;
              return m < kMaxFrames ? s_frame[m] : und_frame(p, k0, th + m * p.dtb);
            },
            [&](bool rho, int i, int j, int k, const T* f, T jx, T jy, T jz, T q) {
              far_deposit(a, i0, j0, k0, i, j, k);
              if (kF32) {
                if (rho)
                  deposit_rho_fixed(p, sRh, sRl, src, i0, j0, k0, i, j, k, f[0], f[1], f[2], sb);
                else
                  deposit_cic(p, src, i, j, k, f[0], f[1], f[2], jx, jy, jz, (T)0);
              } else if (rho) {
                deposit_tile<true>(p, sJ, src, i0, j0, k0, i, j, k, f[0], f[1], f[2], jx, jy, jz,
                                   q);
              } else {
                deposit_tile<false>(p, sJ, src, i0, j0, k0, i, j, k, f[0], f[1], f[2], jx, jy, jz,
                                    q);
              }
            },
            [&]() { return *sl_cell; },
            [&](T* f, U* u) {
              f[0] = sl_f[0]; f[1] = sl_f[kPushThreads]; f[2] = sl_f[2 * kPushThreads];
              u[0] = sl_u[0]; u[1] = sl_u[kPushThreads]; u[2] = sl_u[2 * kPushThreads];
            },
            [&]() { return *sl_id; },
            [&]() {
              if (q + kPushThreads < end)
                prefetch(P, perm, *sl_pos, q + 2 * kPushThreads, end);
            });
      }
      __syncthreads();
      // add the block to the global sources (touched vertices only)
      if (kF32) {
        const float s1 = (float)p.qV * __int_as_float((127 - bsh) << 23);
        const float s2 = s1 * __int_as_float((127 - bsh) << 23);
        for (int c = tid; c < kTPC; c += blockDim.x) {
          const int h = sRh[c], l = sRl[c];
          if (h != 0 || l != 0) {
            const int a = c % kTP, b = (c / kTP) % kTP, cc = c / (kTP * kTP);
            atomicAdd(&src[cidx(i0 - 1 + a, j0 - 1 + b, k0 - 1 + cc, p.nx, p.nxy)].w,
                      (T)((float)h * s1 + (float)l * s2));
          }
        }
      } else {
        for (int c = tid; c < kTPC; c += blockDim.x) {
          const V4<T> v = v4(sJ[c], sJ[kTPC + c], sJ[2 * kTPC + c], sJ[3 * kTPC + c]);
          if (v.x != (T)0 || v.y != (T)0 || v.z != (T)0 || v.w != (T)0) {
            const int a = c % kTP, b = (c / kTP) % kTP, cc = c / (kTP * kTP);
            dep_add(src + cidx(i0 - 1 + a, j0 - 1 + b, k0 - 1 + cc, p.nx, p.nxy), v.x, v.y, v.z,
                    v.w);
          }
        }
      }
      __syncthreads();
    }
  };
  auto sparse = [&](const PushArgs<T, U>& a, int ntiles, double th) {
    const PicP<T>& p = a.p;
    StepState* const& st = a.st;
    const V4<T>* const& pn = a.pn;
    const V4<T>* const& D = a.D;
    V4<T>* const& src = a.src;
    const Parts<T, U>& P = a.P;
    const Parts<T, U>& O = a.O;
    const int* const& perm = a.perm;
    const int* const& offset = a.offset;
    const int* const& tiles = a.tiles;
    int* const& count = a.count;
    int* const& key = a.key;
    int* const& rank = a.rank;
    long long* const& lost_ctr = a.lost_ctr;
    const long long& np = a.np;
    // Sparse tiles: one warp per tile, no staging -- E and B evaluated at the
    // vertices from global memory and the deposits added with global atomics.
    // The whole CTA has left the loop above, so the E/B area is free for the
    // warps' undulator frames.
    const int nsparse = st->n_sparse;
    if (nsparse > 0) {
      const int lane = tid & 31;
      UndFrame<T>* wf = reinterpret_cast<UndFrame<T>*>(sE) + (tid >> 5) * kMaxFrames;
      for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(&st->work_sparse, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= nsparse) break;
        const int tile = tiles[ntiles + w];
        int i0, j0, k0;
        tile_origin(p, tile, &i0, &j0, &k0);
        if (lane < 27) mark_tile(a, tile, lane);
        __syncwarp();
        for (int m = lane; m < p.n_sub && m < kMaxFrames; m += 32)
          wf[m] = und_frame(p, k0, th + m * p.dtb);
        __syncwarp();
        const int beg = offset[tile], end = offset[tile + 1];
        for (int q = beg + lane; q < end; q += 32) {
          const long long pos = perm[q];
          tile_particle<kOpt>(
              p, O, q, count, key, rank, lost_ctr,
              [&](int ci, int cj, int ck, const T* ff, T* E, T* B) {
                gather_eb<kLo>(p, pn, D, ci, cj, ck, ff[0], ff[1], ff[2], E, B);
              },
              [&](int m, int kc, int* kref) {
                *kref = k0;
                return m < kMaxFrames ? wf[m] : und_frame(p, k0, th + m * p.dtb);
              },
              [&](bool rho, int i, int j, int k, const T* f, T jx, T jy, T jz, T q) {
                far_deposit(a, i0, j0, k0, i, j, k);
                deposit_cic(p, src, i, j, k, f[0], f[1], f[2], jx, jy, jz, q);
              },
              [&]() { return P.cell[pos]; },
              [&](T* f, U* u) {
                f[0] = P.fx[pos]; f[1] = P.fy[pos]; f[2] = P.fz[pos];
                u[0] = P.ux[pos]; u[1] = P.uy[pos]; u[2] = P.uz[pos];
              },
              [&]() { return P.id[pos]; },
              [&]() {});
        }
      }
    }
    // particles lost before this step sit at the tail of the sorted order (the
    // bucket after the last tile); they keep that bucket in the re-sort
    lost_tail(a);
  };
  if constexpr (!kBatch) {
    const PushArgs<T, U>& a = prm.args;
    clear_flags(a);
    const int ntiles = a.st->n_tiles;
    const double th = a.p.t0 + ((double)a.st->n + 0.5) * a.p.dt;
    for (;;) {  // the CTA takes tiles from the list until none is left
      if (tid == 0) s_tile = atomicAdd(&a.st->work, 1);
      __syncthreads();
      const int t = s_tile;
      if (t >= ntiles) break;
      dense(a, &prm.tm_pn, &prm.tm_d, t, th);
    }
    sparse(a, ntiles, th);
  } else {
    // the group's non-empty tiles (the dense and the sparse entries of each
    // member's list, all staged) from one counter
    const int M = prm.M;
    for (int r = 0; r < M; ++r) clear_flags(prm.m[r]);
    for (;;) {
      if (tid == 0) s_tile = atomicAdd(prm.work, 1);
      __syncthreads();
      const int w = s_tile;
      if (w >= prm.pref[M]) break;
      const int mi = member_of_tile(prm.pref, M, w);
      const PushArgs<T, U>& a = prm.m[mi];
      const double th = a.p.t0 + ((double)a.st->n + 0.5) * a.p.dt;
      dense(a, &prm.box[mi], &prm.box_d[mi], w - prm.pref[mi], th);
    }
    // the particles each member lost before this step keep their bucket
    for (int r = 0; r < M; ++r) lost_tail(prm.m[r]);
  }
}

}  // namespace mithra
