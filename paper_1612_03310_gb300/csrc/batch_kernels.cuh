// batch_kernels.cuh -- one field step of many simulations of uneven size in
// a fixed handful of launches: every phase of the step (boundary rest,
// potential update, power sample, particle step, the two scan passes of the
// re-sort, the slot map) is one kernel over a work list that spans all
// members, instead of one launch per member and phase.  The members share
// the precision form and the undulator type (the template arguments); each
// member's sizes, coefficients, buffers and tensor maps sit in a device
// table (BatchMember, BatchMaps) written by the host once per membership and
// step parity.
//
// Work lists: the flat phases number their blocks member after member, and
// a block finds its member by binary search in the table's prefix of block
// counts (blk[phase][m] .. blk[phase][m+1]); the particle step is persistent
// (one CTA set for the device) and walks the members' dense tile lists in
// turn, each CTA starting at its own member, taking tiles from a member's
// counter until that member is done, then the sparse lists, then the lost
// tails.
#pragma once
#include "common.cuh"
#include "field_kernels.cuh"
#include "particle_kernels.cuh"
#include "batch_table.cuh"
#include "tile_push.cuh"

namespace mithra {

enum BatchPhase { kBPMur = 0, kBPZ, kBPPow, kBPScan, kBPSlot, kBPCount };

// Member of flat block g: the m with blk[m] <= g < blk[m+1] (blk has M + 1
// non-decreasing entries, blk[0] = 0).
__device__ inline int member_of(const int* __restrict__ blk, int M, int g) {
  int lo = 0, hi = M - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blk[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The member's table entry in shared memory (one copy per block, the hot
// loops read their coefficients from there instead of from global memory).
template <typename X>
__device__ inline void copy_to_shared(X* dst, const X* src) {
  static_assert(sizeof(X) % 4 == 0, "word copy");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int w = threadIdx.x + threadIdx.y * blockDim.x; w < (int)(sizeof(X) / 4);
       w += blockDim.x * blockDim.y)
    d[w] = s[w];
}

// Arguments of the boundary and potential-update phases of a group of
// members, in the launch's parameter space (read where used, like the
// single-simulation kernels' parameters): blk[g] numbers the group's blocks
// member after member.
template <typename T>
struct ZMember {
  StencilP<T> sp;
  const V4<T>* P0;
  const LoV4* L0;
  V4<T>* P1;
  LoV4* L1;
  V4<T>* D;
  V4<T>* S;
  int lz;
  int fused_mur;
};

constexpr int kZGroup = 96;  // 96 x 256 B (FP64) of the 32 KB parameter space

template <typename T>
struct ZParams {
  ZMember<T> m[kZGroup];
  const int* blk;  // blk[0 .. M]
  int M;
};

// Boundary rest (the vertices k_potential_zloop_mur1 leaves), or every
// boundary vertex of members without the fused Mur.
template <bool kLo, typename T>
__global__ void __launch_bounds__(256) kb_mur(const __grid_constant__ ZParams<T> prm) {
  const int g = blockIdx.x;
  const int mi = member_of(prm.blk, prm.M, g);
  const ZMember<T>& m = prm.m[mi];
  const StencilP<T>& p = m.sp;
  const long long t = (long long)(g - prm.blk[mi]) * blockDim.x + threadIdx.x;
  int i, j, k;
  if (m.fused_mur) {
    if (!rest_vertex_at(t, p.nx, p.ny, p.nz, &i, &j, &k)) return;
  } else {
    // every boundary vertex: z faces, y faces (planes 1 .. nz-2), x faces
    const long long nxy = p.nxy;
    long long r = t;
    if (r < 2 * nxy) {
      const long long q = r % nxy;
      i = (int)(q % p.nx); j = (int)(q / p.nx); k = r < nxy ? 0 : p.nz - 1;
    } else if ((r -= 2 * nxy) < 2LL * p.nx * (p.nz - 2)) {
      const long long f = (long long)p.nx * (p.nz - 2), q = r % f;
      i = (int)(q % p.nx); k = 1 + (int)(q / p.nx); j = r < f ? 0 : p.ny - 1;
    } else if ((r -= 2LL * p.nx * (p.nz - 2)) < 2LL * (p.ny - 2) * (p.nz - 2)) {
      const long long f = (long long)(p.ny - 2) * (p.nz - 2), q = r % f;
      j = 1 + (int)(q % (p.ny - 2)); k = 1 + (int)(q / (p.ny - 2)); i = r < f ? 0 : p.nx - 1;
    } else {
      return;
    }
  }
  mur_vertex<kLo, T, true>(p, m.P0, m.L0, m.P1, m.L1, m.D, m.S, i, j, k);
}

// Boundary vertices of a member: the rest of the fused form, or all of them.
__host__ __device__ inline long long batch_mur_count(int nx, int ny, int nz, int fused) {
  return fused ? rest_count(nx, ny, nz)
               : 2LL * nx * ny + 2LL * nx * (nz - 2) + 2LL * (ny - 2) * (nz - 2);
}

// Potential update: block g is the member's (bx, by, bz) column tile and
// plane run, in the register z-marching form.
// (kMur: the members' first-order Mur at the x faces inside the loop; the
// members of a fused batch share the boundary order.)
template <bool kLo, typename T, bool kMur>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (kLo ? 3 : 4) : (kLo ? 1 : 2))
    kb_potential(const __grid_constant__ ZParams<T> prm) {
  const int g = blockIdx.x;
  const int mi = member_of(prm.blk, prm.M, g);
  const ZMember<T>& m = prm.m[mi];
  const int tx = (m.sp.nx + 31) / 32, ty = (m.sp.ny + 7) / 8;
  const int lb = g - prm.blk[mi];
  const int bx = lb % tx, by = (lb / tx) % ty, bz = lb / (tx * ty);
  zloop_body<kLo, T, kMur>(m.sp, m.P0, m.L0, m.P1, m.L1, m.D, m.S, m.lz, bx, by, bz);
}

// Power sample: 64 blocks per recording member.
constexpr int kBatchPowerBlocks = 64;

template <typename T, typename U>
__global__ void __launch_bounds__(256) kb_power(const BatchMember<T, U>* __restrict__ mem,
                                                const int* __restrict__ blk, int M) {
  __shared__ PicP<T> pp;
  const int g = blockIdx.x;
  const int mi = member_of(blk, M, g);
  copy_to_shared(&pp, &mem[mi].pp);
  __syncthreads();
  const BatchMember<T, U>& m = mem[mi];
  power_body(pp, m.P1, m.D, m.power_plane, m.g0, m.b0, m.power_acc, m.st, m.power_end, 1,
             &m.st->err, g - blk[mi], kBatchPowerBlocks);
}

// The particle step of every member is k_push_tiled<.., kBatch = true>
// (tile_push.cuh): persistent CTAs take every member's non-empty tiles from
// one counter; kb_tile_prefix numbers those tiles member after member (from
// the tile counts the last re-sort left) and clears the counter.
template <typename T, typename U>
__global__ void __launch_bounds__(1024) kb_tile_prefix(const BatchMember<T, U>* __restrict__ mem,
                                                       int M, int* __restrict__ pref,
                                                       int* __restrict__ work) {
  __shared__ int ws[32];
  int base = 0;
  for (int c0 = 0; c0 < M; c0 += blockDim.x) {
    const int m = c0 + threadIdx.x;
    int n = 0;
    if (m < M) {
      const StepState* st = mem[m].st;
      n = st->n_tiles + st->n_sparse;
    }
    int tot;
    const int ex = block_exclusive_scan(n, ws, &tot);
    if (m < M) pref[m] = base + ex;
    base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pref[M] = base;
    *work = 0;
  }
}

// First pass of every member's re-sort scan.
template <typename T, typename U>
__global__ void __launch_bounds__(kScanBlock) kb_scan_partials(
    const BatchMember<T, U>* __restrict__ mem, const int* __restrict__ blk, int M) {
  const int g = blockIdx.x;
  const int mi = member_of(blk, M, g);
  const BatchMember<T, U>& m = mem[mi];
  scan_partials_body(m.count, m.nkeys, m.sparse_below, m.scan_part, g - blk[mi]);
}

// Second pass (advances every member's step counter).
template <typename T, typename U>
__global__ void __launch_bounds__(kScanBlock) kb_scan_final(
    const BatchMember<T, U>* __restrict__ mem, const int* __restrict__ blk, int M) {
  const int g = blockIdx.x;
  const int mi = member_of(blk, M, g);
  const BatchMember<T, U>& m = mem[mi];
  scan_final_body(m.count, m.offset, m.tiles, m.nkeys, m.sparse_below, m.scan_part, m.scan_nb,
                  m.st, 1, g - blk[mi]);
}

// The re-sort's slot map (slot_one), 256 particles per block.
template <typename T, typename U>
__global__ void __launch_bounds__(256) kb_slot_map(const BatchMember<T, U>* __restrict__ mem,
                                                  const int* __restrict__ blk, int M) {
  const int g = blockIdx.x;
  const int mi = member_of(blk, M, g);
  const BatchMember<T, U>& m = mem[mi];
  const long long q = (long long)(g - blk[mi]) * blockDim.x + threadIdx.x;
  if (q >= m.np) return;
  slot_one(q, m.key, m.rank, m.offset, m.perm);
}

}  // namespace mithra
