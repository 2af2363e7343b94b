// mithra.cu -- host side of the C ABI declared in include/mithra.h:
// validation, device memory, kernel launch order of one field step, copy-in
// and copy-out.  The kernels live in field_kernels.cuh and
// particle_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "mithra.h"
#include "common.cuh"
#include "field_kernels.cuh"
#include "particle_kernels.cuh"
#include "tile_push.cuh"
#include "diag.cuh"
#include "batch_kernels.cuh"

using namespace mithra;

namespace {
thread_local std::string g_thread_err;
}

namespace mithra {
void set_thread_error(const std::string& msg) { g_thread_err = msg; }
}

struct mithra_sim {
  mithra_grid g{};
  mithra_undulator u{};
  int prec = 1;
  double q_macro = 0.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // the plane diagnostics (power, spectrum) of a step run on a side stream
  // beside the particle step, forked after the potential update and joined
  // before the re-sort advances the step counter
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // inside a captured run of steps, the re-sort of a step (scan and slot
  // map) runs on the side stream beside the next step's potential update,
  // which reads nothing it writes, and is joined before the next particle
  // step; resort_pending marks a step whose re-sort is still to be launched
  // (never true between API calls)
  cudaEvent_t ev_rs_fork = nullptr, ev_rs_join = nullptr;
  bool resort_pending = false;
  int cur = 0;  // P[cur] holds the newest level
  int pb = 0;   // particle buffer in use
  void* P[2] = {nullptr, nullptr};  // psi ping-pong; P[cur] is the newest level
  void* D = nullptr;                // increment newest - previous level
  void* S = nullptr;
  void* PL[2] = {nullptr, nullptr};  // lo parts of the compensated levels (P32_C, P32_U64)
  // particles: pbuf[pb] holds them at the positions perm gives for the
  // slots of the tile order (perm[slot] = position); the particle step
  // writes them to pbuf[1 - pb] in slot order, and the re-sort writes the
  // next perm
  void* pbuf[2] = {nullptr, nullptr};
  int* perm = nullptr;
  int* key = nullptr;
  int* rank = nullptr;
  int* count = nullptr;
  int* offset = nullptr;
  int* tiles = nullptr;  // non-empty tile list written by the scan
  // source-tile flags of the two level parities (StencilP::dirty), each
  // dirty_words words
  unsigned char* dirty = nullptr;
  int dirty_words = 0;
  int4* scan_part = nullptr;  // block sums of the two-pass scan
  StepState* dstate = nullptr;
  double* d_scalar = nullptr;   // one-off reductions
  double* d_power_rec = nullptr;
  int64_t power_cap = 0;
  int64_t power_first = 0;
  int32_t power_plane = 0;
  SeedP seed{};                     // TF/SF seed (seed.on = 0: none)
  // bunch sampling every bunch_every steps into d_bunch_rec (15 doubles each)
  int32_t bunch_every = 0;
  double bunch_kb = 0.0;
  int64_t bunch_first = 0, bunch_cap = 0;
  double* d_bunch_rec = nullptr;
  double* d_bunch_part = nullptr;
  // frequency-resolved power: running Fourier sums at one plane
  int32_t spec_plane = 0;
  int32_t spec_nf = 0;
  double* d_spec_omega = nullptr;
  double* d_spec_acc = nullptr;
  double* d_spec_out = nullptr;
  long long* d_spec_samples = nullptr;
  int64_t np = 0;
  int ntx = 0, nty = 0, ntz = 0, nkeys = 0;
  int64_t n_issued = 0;
  // two steps captured as a CUDA graph, one per parity of the level
  // ping-pong at its start (index cur); dropped when a launch parameter
  // changes
  cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
  double t0 = 0.0;
  // pinned mirror of the device's lost counter and error word, refreshed
  // at the end of every mithra_step and read by the next one
  struct Mirror {
    long long n_lost;
    int err;
  }* h_mirror = nullptr;
  bool strict_lost = false;  // mithra_set_lost_policy
  long long lost_base = 0;   // lost count when strict mode was switched on
  std::string err;
  // potential-update variant: 0 direct, 1 z-marching TMA tiles (needs tm)
  int stencil_variant = 0;
  int lz = 0;  // planes per CTA of the marching form
  int march_resident = 608;  // marching CTAs resident on the device at once
  bool have_tm = false;
  CUtensorMap tm[2];      // psi buffers, plane boxes of the marching update
  CUtensorMap tm_box[2];  // psi buffers, 11^3 boxes of the tiled particle step
  CUtensorMap tm_box_d;   // increment, 11^3 boxes
  CUtensorMap tm_col_d;   // increment, 32 x 8 column boxes of the marching update
  CUtensorMap tm_col_s;   // sources, 32 x 8 column boxes
  int push_variant = 0;   // 0 per-particle, 1 tiled (needs the box maps)
  int push_grid = 0;      // persistent CTAs of the tiled particle step
  int push_max_per_sm = 1;
  int push_ctas_per_sm = 0;
  int push_sparse_below = 0;  // tiles with fewer particles take the per-warp path
  int n_sm = 152;
  mithra_batch* in_batch = nullptr;  // the batch that steps this sim, if any
  // per-kernel event timing
  bool profiling = false;
  struct Rec { int kernel; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> spare;
  double prof_ms[8] = {0};
  int64_t prof_n[8] = {0};
};

void batch_mark_dirty(mithra_batch* b);  // defined with the batch

namespace {

enum KernelId { K_POTENTIAL = 0, K_POWER, K_PUSH, K_SCAN, K_SLOT_MAP, K_SPECTRUM, K_COUNT };
const char* kKernelNames[K_COUNT] = {"potential_step", "power", "push", "scan_counts", "slot_map",
                                     "spectrum"};

cudaEvent_t take_event(mithra_sim* s) {
  if (!s->spare.empty()) {
    cudaEvent_t e = s->spare.back();
    s->spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with an event pair when profiling is on.
struct ProfScope {
  mithra_sim* s;
  int k;
  cudaEvent_t b = nullptr;
  ProfScope(mithra_sim* sim, int kernel) : s(sim), k(kernel) {
    if (!s->profiling) return;
    cudaEvent_t a = take_event(s);
    b = take_event(s);
    cudaEventRecord(a, s->stream);
    s->recs.push_back({k, a, b});
  }
  ~ProfScope() {
    if (b) cudaEventRecord(b, s->stream);
  }
};

void flush_profile(mithra_sim* s) {
  for (auto& r : s->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      s->prof_ms[r.kernel] += ms;
      s->prof_n[r.kernel] += 1;
    }
    s->spare.push_back(r.a);
    s->spare.push_back(r.b);
  }
  s->recs.clear();
}

mithra_status fail(mithra_sim* s, mithra_status st, const std::string& msg) {
  if (s)
    s->err = msg;
  else
    g_thread_err = msg;
  return st;
}

mithra_status cuda_fail(mithra_sim* s, cudaError_t e, const char* where) {
  return fail(s, MITHRA_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define MCHECK(sim, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(sim, e_, #call); \
  } while (0)

size_t real_size(int prec) { return prec == MITHRA_P64 ? sizeof(double) : sizeof(float); }
size_t mom_size(int prec) {
  return (prec == MITHRA_P32 || prec == MITHRA_P32_C) ? sizeof(float) : sizeof(double);
}
// compensated (hi + lo) potential levels
bool has_lo(int prec) { return prec == MITHRA_P32_C || prec == MITHRA_P32_U64; }

// Calls f with null pointers whose pointee types are the field / fraction
// type T and the momentum type U of the precision mode.
template <typename F>
mithra_status with_types(int prec, F&& f) {
  if (prec == MITHRA_P64) return f((double*)nullptr, (double*)nullptr);
  if (prec == MITHRA_P32_U64) return f((float*)nullptr, (FF2*)nullptr);
  return f((float*)nullptr, (float*)nullptr);
}
#define TYPES_OF(t, u)                                   \
  using T = std::remove_pointer_t<decltype(t)>;          \
  using U = std::remove_pointer_t<decltype(u)>

int64_t ncell_of(const mithra_grid* g) { return (int64_t)g->nx * g->ny * g->nz; }

void tiles_of(const mithra_grid* g, int* ntx, int* nty, int* ntz) {
  *ntx = (g->nx + kTile - 1) / kTile;
  *nty = (g->ny + kTile - 1) / kTile;
  *ntz = (g->nz + kTile - 1) / kTile;
}

// bytes of one particle buffer: cell, 3 fractions, 3 momenta, id
size_t particle_buffer_bytes(int64_t np, int prec) {
  return (size_t)np * (2 * sizeof(int) + 3 * real_size(prec) + 3 * mom_size(prec)) + 8 * 256;
}

mithra_status check_grid(const mithra_grid* g, std::string* why) {
  if (!g) { *why = "grid is NULL"; return MITHRA_EINVAL; }
  if (g->nx < 4 || g->ny < 4 || g->nz < 4) { *why = "nx, ny, nz must be >= 4"; return MITHRA_EINVAL; }
  if ((int64_t)g->nx * g->ny * g->nz >= (int64_t)1 << 31) { *why = "grid has >= 2^31 vertices"; return MITHRA_EINVAL; }
  {
    const int64_t tiles = (int64_t)((g->nx + kTile - 1) / kTile) * ((g->ny + kTile - 1) / kTile) *
                          ((g->nz + kTile - 1) / kTile);
    if (tiles + 1 > (int64_t)kScanBlock * kScanBlock) { *why = "grid has too many 8^3 tiles (> 2^20)"; return MITHRA_EINVAL; }
  }
  if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0) || !(g->dt > 0)) { *why = "dx, dy, dz, dt must be > 0"; return MITHRA_EINVAL; }
  if (g->n_sub < 1) { *why = "n_sub must be >= 1"; return MITHRA_EINVAL; }
  if (g->stencil != 0 && g->stencil != 1) { *why = "stencil must be 0 (NSFD) or 1 (standard)"; return MITHRA_EINVAL; }
  if (g->boundary != 1 && g->boundary != 2) {
    *why = "boundary must be 1 (first-order Mur) or 2 (second-order Mur)";
    return MITHRA_EINVAL;
  }
  const double cdt = kC * g->dt;
  const double rx2 = (cdt / g->dx) * (cdt / g->dx), ry2 = (cdt / g->dy) * (cdt / g->dy),
               rz2 = (cdt / g->dz) * (cdt / g->dz);
  if (g->stencil == 0) {
    if (rx2 + ry2 >= 1.0 || rz2 > 1.0 + 1e-12) {
      *why = "NSFD stability needs (c dt/dx)^2 + (c dt/dy)^2 < 1 and c dt <= dz";
      return MITHRA_EUNSTABLE;
    }
  } else if (rx2 + ry2 + rz2 >= 1.0) {
    *why = "standard scheme stability needs c dt < 1/sqrt(1/dx^2 + 1/dy^2 + 1/dz^2)";
    return MITHRA_EUNSTABLE;
  }
  return MITHRA_OK;
}

template <typename T>
StencilP<T> make_stencil(const mithra_grid& g) {
  StencilP<T> p{};
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz;
  p.nxy = (long long)g.nx * g.ny;
  const double cdt = kC * g.dt;
  const double rx2 = (cdt / g.dx) * (cdt / g.dx), ry2 = (cdt / g.dy) * (cdt / g.dy),
               rz2 = (cdt / g.dz) * (cdt / g.dz);
  double A = 0.0;
  if (g.stencil == 0) {
    const double qx = g.dz / g.dx, qy = g.dz / g.dy;
    A = 0.25 * (1.0 + 0.02 / (qx * qx + qy * qy));  // Eq. NSFDCoefficient
  }
  p.rxA = (T)(rx2 * A);
  p.rxB = (T)(rx2 * (1.0 - 2.0 * A));
  p.ryA = (T)(ry2 * A);
  p.ryB = (T)(ry2 * (1.0 - 2.0 * A));
  p.rz2 = (T)rz2;
  p.sA = (T)(cdt * cdt * kMu0);
  p.sphi = (T)(cdt * cdt / kEps0);
  for (int m = 0; m < 8; ++m) {
    double d2 = 0.0;
    if (m & 1) d2 += g.dx * g.dx;
    if (m & 2) d2 += g.dy * g.dy;
    if (m & 4) d2 += g.dz * g.dz;
    const double d = std::sqrt(d2);
    p.mb0[m] = (T)((cdt - d) / (cdt + d));
  }
  const double dd[3] = {g.dx, g.dy, g.dz};
  const int tang[3][2] = {{1, 2}, {0, 2}, {0, 1}};
  for (int a = 0; a < 3; ++a)
    for (int t = 0; t < 2; ++t) {
      const double r = cdt / dd[tang[a][t]];
      p.m2[a][t] = (T)(r * r * dd[a] / (2.0 * (cdt + dd[a])));
    }
  p.mur2 = g.boundary == 2 ? 1 : 0;
  p.space_charge = g.space_charge ? 1 : 0;
  return p;
}

template <typename T>
PicP<T> make_pic(const mithra_sim* s) {
  const mithra_grid& g = s->g;
  const mithra_undulator& u = s->u;
  PicP<T> p{};
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz;
  p.nxy = (long long)g.nx * g.ny;
  p.x0 = g.x0; p.y0 = g.y0; p.z0 = g.z0;
  p.dxd = g.dx; p.dyd = g.dy; p.dzd = g.dz;
  p.inv2dx = (T)(0.5 / g.dx); p.inv2dy = (T)(0.5 / g.dy); p.inv2dz = (T)(0.5 / g.dz);
  p.inv4dx = (T)(0.25 / g.dx); p.inv4dy = (T)(0.25 / g.dy); p.inv4dz = (T)(0.25 / g.dz);
  p.invdt = (T)(1.0 / g.dt);
  const double qm = -kQe / kMe;  // electrons
  const double dtb = g.dt / g.n_sub;
  p.h = qm * dtb / (2.0 * kC);
  p.an = qm * dtb / 2.0;
  p.h_hi = (float)p.h; p.h_lo = (float)(p.h - (double)p.h_hi);
  p.an_hi = (float)p.an; p.an_lo = (float)(p.an - (double)p.an_hi);
  p.cx = (T)(kC * dtb / g.dx); p.cy = (T)(kC * dtb / g.dy); p.cz = (T)(kC * dtb / g.dz);
  p.n_sub = g.n_sub;
  p.t0 = s->t0; p.dt = g.dt; p.dtb = dtb;
  p.und_type = u.type == 1 ? 1 : 0;
  p.und_on = (u.type == 1) ? (u.a0 != 0.0) : (u.K != 0.0);
  p.fringe = u.fringe ? 1 : 0;
  p.g0 = u.gamma0;
  const double b0 = std::sqrt(1.0 - 1.0 / (u.gamma0 * u.gamma0));
  if (p.und_type == 1) {
    // optical plane wave: tau of a rest-frame event, the signal constants,
    // and the rest-frame field per unit s' (E_perp = gamma0 (E' + v x B'),
    // B_perp = gamma0 (B' - v x E'/c^2) of E' = -p A0 s', B' = -(d/c) z x p A0 s')
    const double d = u.direction < 0 ? -1.0 : 1.0;
    const double pn = std::sqrt(u.pol_x * u.pol_x + u.pol_y * u.pol_y);
    const double px = u.pol_x / pn, py = u.pol_y / pn;
    const double A0 = u.a0 * kMe * kC / kQe;
    const double tv = u.variance / kC;
    p.osig = u.signal;
    p.w0_d = 2.0 * kPi * kC / u.lambda_l;
    p.cep = u.cep;
    p.t0o = u.offset / kC;
    p.tau_t = u.gamma0 * (1.0 - d * b0);
    p.tau_z = u.gamma0 * (b0 - d) / kC;
    p.tau_c = d * u.z0_lab / kC;
    p.w0 = (T)p.w0_d;
    p.env_a = (T)(2.0 * std::log(2.0) / (tv * tv));
    p.inv_tv = (T)(1.0 / tv);
    p.oex = (T)(-u.gamma0 * (1.0 - d * b0) * A0 * px);
    p.oey = (T)(-u.gamma0 * (1.0 - d * b0) * A0 * py);
    p.obx = (T)(u.gamma0 * (d - b0) * A0 * py / kC);
    p.oby = (T)(-u.gamma0 * (d - b0) * A0 * px / kC);
    p.dtau_cell = (T)(p.tau_z * g.dz);
  }
  p.b0c = b0 * kC;
  p.zent = u.z_ent_lab;
  p.L = u.length_lab;
  p.lam_u = u.lambda_u;
  p.inv_lam_u = 1.0 / u.lambda_u;
  p.ku_d = 2.0 * kPi / u.lambda_u;
  p.ku = (T)p.ku_d;
  p.B0 = (T)(2.0 * kPi * kMe * kC * u.K / (kQe * u.lambda_u));
  p.ex_fac = (T)(-u.gamma0 * b0 * kC);
  p.by_fac = (T)u.gamma0;
  p.g0dz = (T)(u.gamma0 * g.dz);
  p.y0f = (T)g.y0;
  p.dyf = (T)g.dy;
  const double V = g.dx * g.dy * g.dz;
  p.qV = (T)(s->q_macro / V);
  p.jx = (T)(s->q_macro / V * g.dx / g.dt);
  p.jy = (T)(s->q_macro / V * g.dy / g.dt);
  p.jz = (T)(s->q_macro / V * g.dz / g.dt);
  p.ntx = s->ntx; p.nty = s->nty; p.ntz = s->ntz; p.nkeys = s->nkeys;
  p.fd_nx = make_fastdiv(g.nx);
  p.fd_nxy = make_fastdiv(g.nx * g.ny);
  return p;
}

template <typename T, typename U>
Parts<T, U> parts_of(mithra_sim* s, int b) {
  Parts<T, U> P{};
  char* base = static_cast<char*>(s->pbuf[b]);
  auto carve = [&](size_t bytes) {
    char* r = base;
    base += (bytes + 255) & ~size_t(255);
    return r;
  };
  const size_t n = (size_t)s->np;
  P.cell = reinterpret_cast<int*>(carve(n * sizeof(int)));
  P.fx = reinterpret_cast<T*>(carve(n * sizeof(T)));
  P.fy = reinterpret_cast<T*>(carve(n * sizeof(T)));
  P.fz = reinterpret_cast<T*>(carve(n * sizeof(T)));
  P.ux = reinterpret_cast<U*>(carve(n * sizeof(U)));
  P.uy = reinterpret_cast<U*>(carve(n * sizeof(U)));
  P.uz = reinterpret_cast<U*>(carve(n * sizeof(U)));
  P.id = reinterpret_cast<int*>(carve(n * sizeof(int)));
  return P;
}

// Two-pass scan of the per-tile counts (see k_scan_final), on stream q
// (default: the simulation's).
void launch_scan(mithra_sim* s, int advance, cudaStream_t q = nullptr) {
  if (!q) q = s->stream;
  const int nb = (s->nkeys + 1 + kScanBlock - 1) / kScanBlock;
  const int sparse_below = s->push_variant == 1 ? s->push_sparse_below : 0;
  k_scan_partials<<<nb, kScanBlock, 0, q>>>(s->count, s->nkeys, sparse_below, s->scan_part);
  k_scan_final<<<nb, kScanBlock, 0, q>>>(s->count, s->offset, s->tiles, s->nkeys,
                                                 sparse_below, s->scan_part, nb, s->dstate,
                                                 advance);
}

// Instantiated forms of the particle step: without lo parts (P32, P64) and
// with them (P32_C, P32_U64).
template <typename T, typename U>
constexpr bool push_form_plain() { return sizeof(U) == sizeof(T); }
template <typename T, typename U>
constexpr bool push_form_lo() { return sizeof(T) == 4; }

// Persistent grid of the tiled particle step: as many CTAs as fit on the
// device at once.
template <typename T, typename U>
mithra_status setup_push_grid(mithra_sim* s) {
  const int smem = tile_smem_bytes<T, U>();
  if constexpr (push_form_plain<T, U>()) {
    MCHECK(s, cudaFuncSetAttribute(k_push_tiled<false, T, U>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    MCHECK(s, cudaFuncSetAttribute(k_push_tiled<true, T, U>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  }
  if constexpr (push_form_lo<T, U>()) {
    MCHECK(s, cudaFuncSetAttribute(k_push_tiled<false, T, U, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    MCHECK(s, cudaFuncSetAttribute(k_push_tiled<true, T, U, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  }
  int dev = 0, nsm = 0, per_sm = 0;
  MCHECK(s, cudaGetDevice(&dev));
  MCHECK(s, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if constexpr (push_form_plain<T, U>())
    MCHECK(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_tiled<false, T, U>,
                                                            kPushThreads, smem));
  else
    MCHECK(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &per_sm, k_push_tiled<false, T, U, true>, kPushThreads, smem));
  s->n_sm = nsm;
  s->push_max_per_sm = per_sm > 0 ? per_sm : 1;
  s->push_grid = nsm * s->push_max_per_sm;
  return MITHRA_OK;
}

// Planes per CTA of the marching update: the column tiles times the plane
// runs fill two waves of the CTAs the device holds at once (resident), with
// at least 8 planes per run.
int default_lz(const mithra_grid* g, int resident) {
  const long long tiles = (long long)((g->nx + kMX - 1) / kMX) * ((g->ny + kMY - 1) / kMY);
  long long runs = 2 * resident / tiles;
  if (runs < 1) runs = 1;
  long long lz = (g->nz + runs - 1) / runs;
  if (lz < 8) lz = 8;
  if (lz > g->nz) lz = g->nz;
  return (int)lz;
}

template <typename T>
mithra_status setup_march(mithra_sim* s) {
  MCHECK(s, cudaFuncSetAttribute(k_potential_march<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 march_smem_bytes<T>()));
  int dev = 0, nsm = 0, per_sm = 0;
  MCHECK(s, cudaGetDevice(&dev));
  MCHECK(s, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  MCHECK(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_potential_march<T>,
                                                          kMX * kMY, march_smem_bytes<T>()));
  s->march_resident = nsm * (per_sm > 0 ? per_sm : 1);
  return MITHRA_OK;
}

unsigned blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}

// Marks the sources of both level parities as possibly nonzero anywhere, so
// that the next two potential updates read every vertex's (after writers
// that mark no tiles: the initial deposit, the per-particle step, a set or
// restored source field).
void mark_sources_everywhere(mithra_sim* s) {
  cudaMemsetAsync(reinterpret_cast<char*>(s->dstate) + offsetof(StepState, src_all), 1,
                  sizeof(StepState::src_all), s->stream);
}

// The source-tile flags of level parity c in the stencil parameters.
template <typename T>
void set_source_flags(const mithra_sim* s, int c, StencilP<T>* sp) {
  sp->dirty = s->dirty + (size_t)c * 4 * s->dirty_words;
  sp->src_all = &s->dstate->src_all[c];
  sp->ntx = s->ntx;
  sp->nty = s->nty;
}

// The re-sort of the particle step just launched: scan of the tile counts
// (it advances the device step counter) and the slot map, on stream q.
void launch_resort(mithra_sim* s, cudaStream_t q) {
  {
    ProfScope ps(s, K_SCAN);
    launch_scan(s, 1, q);
  }
  ProfScope ps(s, K_SLOT_MAP);
  k_slot_map<<<blocks_for(s->np, 256 * kSlotPer), 256, 0, q>>>(s->np, s->key, s->rank,
                                                               s->offset, s->perm);
}

// One field step.  defer: leave this step's re-sort to the next launch_step
// of the same captured run, which runs it beside its potential update.
template <typename T, typename U>
mithra_status launch_step(mithra_sim* s, bool defer = false) {
  // the previous step's re-sort, beside this step's potential update (which
  // reads neither the tile counts nor the slot map), joined before the seed
  // and the particle step read the step counter it advances
  const bool overlap = s->resort_pending;
  if (overlap) {
    cudaEventRecord(s->ev_rs_fork, s->stream);
    cudaStreamWaitEvent(s->side, s->ev_rs_fork, 0);
    launch_resort(s, s->side);
    cudaEventRecord(s->ev_rs_join, s->side);
    s->resort_pending = false;
  }
  StencilP<T> sp = make_stencil<T>(s->g);
  set_source_flags(s, s->cur, &sp);
  PicP<T> pp = make_pic<T>(s);
  V4<T>* P0 = static_cast<V4<T>*>(s->P[s->cur]);       // psi^n
  V4<T>* P1 = static_cast<V4<T>*>(s->P[1 - s->cur]);   // receives psi^{n+1}
  LoV4* L0 = static_cast<LoV4*>(s->PL[s->cur]);        // lo parts (compensated levels)
  LoV4* L1 = static_cast<LoV4*>(s->PL[1 - s->cur]);
  pp.plo = L1;  // E and B of this step come from psi^{n+1}
  V4<T>* Dn = static_cast<V4<T>*>(s->D);               // D^{n-1/2} -> D^{n+1/2}
  V4<T>* S = static_cast<V4<T>*>(s->S);
  {
    ProfScope ps(s, K_POTENTIAL);
    // first-order Mur at the x and y faces is fused into the z-marching
    // form (the rest first, by the boundary kernel); the other forms and
    // second-order Mur take the boundary kernel for every boundary vertex
    const bool fused = s->stencil_variant == 2 && s->g.boundary == 1;
    // beside the z-marching form the boundary recomputes D_q^+ in its
    // arithmetic
    const bool zm = s->stencil_variant == 2;
    const dim3 mg = mur_grid(s->g.nx, s->g.ny, s->g.nz);
    const unsigned rg = blocks_for(rest_count(s->g.nx, s->g.ny, s->g.nz), 256);
    if (fused && L0)
      k_mur_boundary<true, T, true, true><<<rg, 256, 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S);
    else if (fused)
      k_mur_boundary<false, T, true, true><<<rg, 256, 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S);
    else if (zm && L0)
      k_mur_boundary<true, T, false, true><<<mg, dim3(32, 8), 0, s->stream>>>(sp, P0, L0, P1, L1,
                                                                             Dn, S);
    else if (zm)
      k_mur_boundary<false, T, false, true><<<mg, dim3(32, 8), 0, s->stream>>>(sp, P0, L0, P1, L1,
                                                                              Dn, S);
    else if (L0)
      k_mur_boundary<true, T><<<mg, dim3(32, 8), 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S);
    else
      k_mur_boundary<false, T><<<mg, dim3(32, 8), 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S);
    if (s->stencil_variant == 2) {
      dim3 blk(32, 8, 1);
      dim3 grd((s->g.nx + 31) / 32, (s->g.ny + 7) / 8, (s->g.nz + s->lz - 1) / s->lz);
      if (L0 && fused)
        k_potential_zloop_mur1<true, T><<<grd, blk, 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S, s->lz);
      else if (L0)
        k_potential_zloop<true, T><<<grd, blk, 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S, s->lz);
      else if (fused)
        k_potential_zloop_mur1<false, T><<<grd, blk, 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S, s->lz);
      else
        k_potential_zloop<false, T><<<grd, blk, 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S, s->lz);
    } else if (s->stencil_variant == 1 && s->have_tm && !L0) {
      dim3 grd((s->g.nx + kMX - 1) / kMX, (s->g.ny + kMY - 1) / kMY,
               (s->g.nz + s->lz - 1) / s->lz);
      k_potential_march<T><<<grd, kMX * kMY, march_smem_bytes<T>(), s->stream>>>(
          s->tm[s->cur], s->tm_col_d, s->tm_col_s, sp, P0, P1, Dn, S, s->lz, &s->dstate->err);
    } else {
      dim3 blk(32, 8, 1);
      dim3 grd((s->g.nx + 31) / 32, (s->g.ny + 7) / 8, s->g.nz);
      if (L0)
        k_potential_step<true, T><<<grd, blk, 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S);
      else
        k_potential_step<false, T><<<grd, blk, 0, s->stream>>>(sp, P0, L0, P1, L1, Dn, S);
    }
    if (overlap) cudaStreamWaitEvent(s->stream, s->ev_rs_join, 0);
    if (s->seed.on && s->seed.beam) {
      dim3 blk(kSeedTile, kSeedTile, 1);
      dim3 grd((s->g.nx - 2 + kSeedTile - 1) / kSeedTile,
               (s->g.ny - 2 + kSeedTile - 1) / kSeedTile, 2);
      if (L0)
        k_seed_tfsf_beam<true, T><<<grd, blk, 0, s->stream>>>(sp, s->seed, s->dstate, P1, L1, Dn);
      else
        k_seed_tfsf_beam<false, T><<<grd, blk, 0, s->stream>>>(sp, s->seed, s->dstate, P1, L1,
                                                                Dn);
    } else if (s->seed.on) {
      dim3 blk(32, 8, 1);
      dim3 grd((s->g.nx - 2 + 31) / 32, (s->g.ny - 2 + 7) / 8, 2);
      if (L0)
        k_seed_tfsf<true, T><<<grd, blk, 0, s->stream>>>(sp, s->seed, s->dstate, P1, L1, Dn);
      else
        k_seed_tfsf<false, T><<<grd, blk, 0, s->stream>>>(sp, s->seed, s->dstate, P1, L1, Dn);
    }
  }
  // with per-kernel timing every kernel stays on the simulation's stream
  const bool branch = !s->profiling && (s->power_cap > 0 || s->spec_nf > 0);
  cudaStream_t dq = s->stream;
  if (branch) {
    cudaEventRecord(s->ev_fork, s->stream);
    cudaStreamWaitEvent(s->side, s->ev_fork, 0);
    dq = s->side;
  }
  if (s->power_cap > 0) {
    ProfScope ps(s, K_POWER);
    k_power<T><<<64, 256, 0, dq>>>(pp, P1, Dn, s->power_plane, s->u.gamma0,
                                          std::sqrt(1.0 - 1.0 / (s->u.gamma0 * s->u.gamma0)),
                                          s->d_power_rec - s->power_first, s->dstate,
                                          s->power_first + s->power_cap, 1, &s->dstate->err);
  }
  if (s->spec_nf > 0) {
    ProfScope ps(s, K_SPECTRUM);
    const double g0 = s->u.gamma0;
    const long long nv = (long long)(s->g.nx - 2) * (s->g.ny - 2);
    k_spectrum_accumulate<T><<<blocks_for(nv, 256), 256, 0, dq>>>(
        pp, P1, Dn, s->spec_plane, g0, std::sqrt(1.0 - 1.0 / (g0 * g0)),
        s->g.z0 + s->spec_plane * s->g.dz, s->dstate, s->spec_nf, s->d_spec_omega,
        s->d_spec_acc, s->d_spec_samples);
  }
  if (s->np > 0) {
    Parts<T, U> A = parts_of<T, U>(s, s->pb), B = parts_of<T, U>(s, 1 - s->pb);
    {
      ProfScope ps(s, K_PUSH);
      const bool opt = pp.und_type == 1;
      const bool lo = L1 != nullptr;
      constexpr bool kAnyLo = !push_form_plain<T, U>();  // a form that exists, for the type
      if (s->push_variant == 1 && s->have_tm) {
        decltype(&k_push_tiled<false, T, U, kAnyLo>) kern = nullptr;
        if constexpr (push_form_plain<T, U>())
          if (!lo) kern = opt ? k_push_tiled<true, T, U> : k_push_tiled<false, T, U>;
        if constexpr (push_form_lo<T, U>())
          if (lo) kern = opt ? k_push_tiled<true, T, U, true> : k_push_tiled<false, T, U, true>;
        if (!kern) return fail(s, MITHRA_EINVAL, "no particle-step form for this precision");
        PushParams<T, U, false> prm;
        prm.tm_pn = s->tm_box[1 - s->cur];
        prm.tm_d = s->tm_box_d;
        PushArgs<T, U>& pa = prm.args;
        pa.p = pp;
        pa.st = s->dstate;
        pa.pn = P1;
        pa.D = Dn;
        pa.src = S;
        pa.P = A;
        pa.O = B;
        pa.perm = s->perm;
        pa.offset = s->offset;
        pa.tiles = s->tiles;
        pa.count = s->count;
        pa.key = s->key;
        pa.rank = s->rank;
        pa.lost_ctr = &s->dstate->n_lost;
        pa.np = s->np;
        pa.dirty = s->dirty;
        pa.dirty_words = s->dirty_words;
        pa.cur = s->cur;
        // a programmatic dependent launch: the grid is scheduled as the
        // work before it drains and waits at its start for that work
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(s->push_grid);
        cfg.blockDim = dim3(kPushThreads);
        cfg.dynamicSmemBytes = tile_smem_bytes<T, U>();
        cfg.stream = s->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t le = cudaLaunchKernelEx(&cfg, kern, prm);
        if (le != cudaSuccess) return cuda_fail(s, le, "particle step launch");
      } else {
        decltype(&k_push<false, T, U, kAnyLo>) kern = nullptr;
        if constexpr (push_form_plain<T, U>())
          if (!lo) kern = opt ? k_push<true, T, U> : k_push<false, T, U>;
        if constexpr (push_form_lo<T, U>())
          if (lo) kern = opt ? k_push<true, T, U, true> : k_push<false, T, U, true>;
        if (!kern) return fail(s, MITHRA_EINVAL, "no particle-step form for this precision");
        kern<<<blocks_for(s->np, 256), 256, 0, s->stream>>>(pp, s->dstate, P1, Dn, S, A, B,
                                                             s->perm, s->np, s->count, s->key,
                                                             s->rank, &s->dstate->n_lost);
        mark_sources_everywhere(s);  // this form marks no tiles
      }
    }
    if (s->bunch_every > 0) {
      ProfScope ps(s, K_SPECTRUM);
      const int nb = (int)std::min<long long>(blocks_for(s->np, 256), 1024);
      k_bunch_partial<T, U><<<nb, 256, 0, s->stream>>>(pp, B, s->np, s->bunch_kb, s->d_bunch_part,
                                                        s->dstate, s->bunch_first, s->bunch_every);
      k_bunch_final<<<1, 32, 0, s->stream>>>(s->d_bunch_part, nb, s->d_bunch_rec, s->dstate,
                                             s->bunch_first, s->bunch_every, s->bunch_cap);
    }
    if (branch) {
      cudaEventRecord(s->ev_join, s->side);
      cudaStreamWaitEvent(s->stream, s->ev_join, 0);
    }
    if (defer && !s->profiling)
      s->resort_pending = true;
    else
      launch_resort(s, s->stream);
    s->pb = 1 - s->pb;
  } else {
    if (branch) {
      cudaEventRecord(s->ev_join, s->side);
      cudaStreamWaitEvent(s->stream, s->ev_join, 0);
    }
    launch_scan(s, 1);
  }
  s->cur = 1 - s->cur;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
  return MITHRA_OK;
}

template <typename T, typename U>
mithra_status init_particles(mithra_sim* s, const mithra_bunch* b) {
  const PicP<T> pp = make_pic<T>(s);
  const int64_t n = s->np;
  double* d = nullptr;
  MCHECK(s, cudaMalloc(&d, sizeof(double) * 6 * (size_t)n));
  const double* src[6] = {b->x, b->y, b->z, b->ux, b->uy, b->uz};
  for (int a = 0; a < 6; ++a)
    MCHECK(s, cudaMemcpyAsync(d + a * n, src[a], sizeof(double) * n, cudaMemcpyHostToDevice,
                              s->stream));
  Parts<T, U> A = parts_of<T, U>(s, 0), B = parts_of<T, U>(s, 1);
  long long* lost = &s->dstate->n_lost;
  k_init_particles<T, U><<<blocks_for(n, 256), 256, 0, s->stream>>>(
      pp, n, d, d + n, d + 2 * n, d + 3 * n, d + 4 * n, d + 5 * n, A, s->count, s->key, s->rank,
      lost);
  launch_scan(s, 0);
  k_sort_particles<T, U><<<blocks_for(n, 256), 256, 0, s->stream>>>(A, B, n, s->key, s->rank,
                                                                    s->offset, s->perm);
  s->pb = 1;
  k_deposit_rho<T, U><<<blocks_for(n, 256), 256, 0, s->stream>>>(pp, B, n,
                                                              static_cast<V4<T>*>(s->S));
  mark_sources_everywhere(s);
  MCHECK(s, cudaGetLastError());
  MCHECK(s, cudaStreamSynchronize(s->stream));
  MCHECK(s, cudaFree(d));
  return MITHRA_OK;
}

// Copies the device's lost counter and error word into the pinned mirror
// (ordered on the stream; read by the next mithra_step).
cudaError_t refresh_mirror(mithra_sim* s) {
  static_assert(offsetof(StepState, err) - offsetof(StepState, n_lost) ==
                    offsetof(mithra_sim::Mirror, err) - offsetof(mithra_sim::Mirror, n_lost),
                "mirror layout");
  return cudaMemcpyAsync(s->h_mirror, &s->dstate->n_lost,
                         offsetof(StepState, err) + sizeof(int) - offsetof(StepState, n_lost),
                         cudaMemcpyDeviceToHost, s->stream);
}

// Waits for the stream; the status of its work.  report_lost: strict mode's
// lost particles count as a failure (mithra_sync, mithra_batch_sync).
mithra_status sync_status(mithra_sim* s, bool report_lost = false) {
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  StepState st;
  e = cudaMemcpy(&st, s->dstate, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(s, e, "state copy");
  if (st.err & 1) return fail(s, MITHRA_ENUMERIC, "NaN or Inf in a power reduction");
  if (report_lost && s->strict_lost && st.n_lost > s->lost_base)
    return fail(s, MITHRA_ELOST, std::to_string(st.n_lost - s->lost_base) +
                                     " particle(s) left the valid region (strict mode)");
  return MITHRA_OK;
}

template <typename T>
mithra_status copy_field_impl(mithra_sim* s, int what, double* out) {
  PicP<T> pp = make_pic<T>(s);
  pp.plo = static_cast<const LoV4*>(s->PL[s->cur]);
  const int64_t n = ncell_of(&s->g);
  double* d = nullptr;
  MCHECK(s, cudaMalloc(&d, sizeof(double) * n));
  const V4<T>* Pn = static_cast<const V4<T>*>(s->P[s->cur]);
  const V4<T>* Po = static_cast<const V4<T>*>(s->P[1 - s->cur]);
  const V4<T>* Dn = static_cast<const V4<T>*>(s->D);
  const V4<T>* lev = Pn;
  const LoV4* levlo = static_cast<const LoV4*>(s->PL[s->cur]);
  int code = 0;
  if (what <= MITHRA_BZ) code = what;
  else if (what <= MITHRA_AZ) code = 6 + (what - MITHRA_AX);
  else if (what <= MITHRA_JZ) code = 10 + (what - MITHRA_JX);
  else if (what == MITHRA_PHI) code = 9;
  else if (what == MITHRA_RHO) code = 13;
  else {
    lev = Po;
    levlo = static_cast<const LoV4*>(s->PL[1 - s->cur]);
    code = 6 + (what - MITHRA_AX_PREV);
  }
  k_extract<T><<<1024, 256, 0, s->stream>>>(pp, Pn, Dn, lev, levlo,
                                            static_cast<const V4<T>*>(s->S), code, d);
  MCHECK(s, cudaGetLastError());
  MCHECK(s, cudaMemcpyAsync(out, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  mithra_status st = sync_status(s);
  cudaFree(d);
  return st;
}

template <typename T>
mithra_status set_field_impl(mithra_sim* s, int what, const double* in) {
  const int64_t n = ncell_of(&s->g);
  V4<T>* dst;
  LoV4* dstlo = nullptr;
  int comp;
  LoV4* Lc = static_cast<LoV4*>(s->PL[s->cur]);
  LoV4* Lp = static_cast<LoV4*>(s->PL[1 - s->cur]);
  if (what >= MITHRA_AX && what <= MITHRA_AZ) { dst = static_cast<V4<T>*>(s->P[s->cur]); dstlo = Lc; comp = what - MITHRA_AX; }
  else if (what == MITHRA_PHI) { dst = static_cast<V4<T>*>(s->P[s->cur]); dstlo = Lc; comp = 3; }
  else if (what >= MITHRA_JX && what <= MITHRA_JZ) { dst = static_cast<V4<T>*>(s->S); comp = what - MITHRA_JX; }
  else if (what == MITHRA_RHO) { dst = static_cast<V4<T>*>(s->S); comp = 3; }
  else if (what >= MITHRA_AX_PREV && what <= MITHRA_PHI_PREV) { dst = static_cast<V4<T>*>(s->P[1 - s->cur]); dstlo = Lp; comp = what - MITHRA_AX_PREV; }
  else return fail(s, MITHRA_EINVAL, "field cannot be set (E and B derive from the potentials)");
  double* d = nullptr;
  MCHECK(s, cudaMalloc(&d, sizeof(double) * n));
  MCHECK(s, cudaMemcpyAsync(d, in, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
  k_insert<T><<<1024, 256, 0, s->stream>>>(n, d, dst, dstlo, comp);
  if (dst == static_cast<V4<T>*>(s->S)) mark_sources_everywhere(s);
  if (dst != static_cast<V4<T>*>(s->S))
    k_increment<T><<<1024, 256, 0, s->stream>>>(n, static_cast<const V4<T>*>(s->P[s->cur]),
                                                static_cast<const V4<T>*>(s->P[1 - s->cur]),
                                                Lc, Lp, static_cast<V4<T>*>(s->D));
  MCHECK(s, cudaGetLastError());
  mithra_status st = sync_status(s);
  cudaFree(d);
  return st;
}

template <typename T>
mithra_status sample_impl(mithra_sim* s, uint32_t mask, const int32_t* ijk, int64_t npts,
                          double* out) {
  PicP<T> pp = make_pic<T>(s);
  pp.plo = static_cast<const LoV4*>(s->PL[s->cur]);
  const int m = __builtin_popcount(mask);
  int* dijk = nullptr;
  double* dout = nullptr;
  MCHECK(s, cudaMalloc(&dijk, sizeof(int) * 3 * npts));
  MCHECK(s, cudaMalloc(&dout, sizeof(double) * m * npts));
  MCHECK(s, cudaMemcpyAsync(dijk, ijk, sizeof(int) * 3 * npts, cudaMemcpyHostToDevice, s->stream));
  k_sample<T><<<blocks_for(npts, 128), 128, 0, s->stream>>>(
      pp, static_cast<const V4<T>*>(s->P[s->cur]), static_cast<const V4<T>*>(s->D),
      static_cast<const V4<T>*>(s->S), dijk, npts, mask, m, dout);
  MCHECK(s, cudaGetLastError());
  MCHECK(s, cudaMemcpyAsync(out, dout, sizeof(double) * m * npts, cudaMemcpyDeviceToHost,
                            s->stream));
  mithra_status st = sync_status(s);
  cudaFree(dijk);
  cudaFree(dout);
  return st;
}

template <typename T>
mithra_status power_impl(mithra_sim* s, int kp, double* p) {
  PicP<T> pp = make_pic<T>(s);
  pp.plo = static_cast<const LoV4*>(s->PL[s->cur]);
  MCHECK(s, cudaMemsetAsync(s->d_scalar, 0, sizeof(double), s->stream));
  const double g0 = s->u.gamma0;
  k_power<T><<<64, 256, 0, s->stream>>>(pp, static_cast<const V4<T>*>(s->P[s->cur]),
                                        static_cast<const V4<T>*>(s->D), kp, g0,
                                        std::sqrt(1.0 - 1.0 / (g0 * g0)), s->d_scalar, s->dstate,
                                        0, 0, &s->dstate->err);
  MCHECK(s, cudaGetLastError());
  MCHECK(s, cudaMemcpyAsync(p, s->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  return sync_status(s);
}

template <typename T, typename U>
mithra_status copy_particles_impl(mithra_sim* s, double* out7) {
  const PicP<T> pp = make_pic<T>(s);
  double* d = nullptr;
  MCHECK(s, cudaMalloc(&d, sizeof(double) * 7 * (size_t)s->np));
  k_copy_out<T, U><<<blocks_for(s->np, 256), 256, 0, s->stream>>>(pp, parts_of<T, U>(s, s->pb),
                                                                  s->np, d);
  MCHECK(s, cudaGetLastError());
  MCHECK(s, cudaMemcpyAsync(out7, d, sizeof(double) * 7 * (size_t)s->np, cudaMemcpyDeviceToHost,
                            s->stream));
  mithra_status st = sync_status(s);
  cudaFree(d);
  return st;
}

template <typename T, typename U>
mithra_status bunch_stats_impl(mithra_sim* s, double kb, double* out14) {
  const PicP<T> pp = make_pic<T>(s);
  const int nb = (int)std::min<long long>(blocks_for(s->np, 256), 1024);
  double* d = nullptr;
  MCHECK(s, cudaMalloc(&d, sizeof(double) * ((size_t)nb * kBunchSums + 14)));
  k_bunch_partial<T, U><<<nb, 256, 0, s->stream>>>(pp, parts_of<T, U>(s, s->pb), s->np, kb, d);
  k_bunch_final<<<1, 32, 0, s->stream>>>(d, nb, d + (size_t)nb * kBunchSums);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out14, d + (size_t)nb * kBunchSums, sizeof(double) * 14,
                        cudaMemcpyDeviceToHost, s->stream);
  mithra_status st = e == cudaSuccess ? sync_status(s) : cuda_fail(s, e, "bunch statistics");
  cudaFree(d);
  return st;
}

void free_spectrum(mithra_sim* s) {
  for (void* p : {(void*)s->d_spec_omega, (void*)s->d_spec_acc, (void*)s->d_spec_out,
                  (void*)s->d_spec_samples})
    if (p) cudaFree(p);
  s->d_spec_omega = s->d_spec_acc = s->d_spec_out = nullptr;
  s->d_spec_samples = nullptr;
  s->spec_nf = 0;
}

void lab_of(const mithra_sim* s, int32_t kp, double t, double* t_lab, double* z_lab) {
  const double g0 = s->u.gamma0;
  const double b0 = std::sqrt(1.0 - 1.0 / (g0 * g0));
  const double zp = s->g.z0 + kp * s->g.dz;
  *t_lab = g0 * (t + b0 * zp / kC);
  *z_lab = g0 * (zp + b0 * kC * t);
}

void free_all(mithra_sim* s) {
  if (s->stream) cudaStreamSynchronize(s->stream);
  void* ptrs[] = {s->P[0], s->P[1], s->PL[0], s->PL[1], s->D, s->S, s->pbuf[0], s->pbuf[1], s->perm, s->key, s->rank, s->count,
                  s->offset, s->tiles, s->dirty, s->scan_part, s->dstate, s->d_scalar, s->d_power_rec,
                  s->d_spec_omega, s->d_spec_acc, s->d_spec_out, s->d_spec_samples,
                  s->d_bunch_rec, s->d_bunch_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->h_mirror) cudaFreeHost(s->h_mirror);
  for (auto& r : s->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : s->spare) cudaEventDestroy(e);
  for (cudaGraphExec_t e : s->step_exec)
    if (e) cudaGraphExecDestroy(e);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->ev_rs_fork) cudaEventDestroy(s->ev_rs_fork);
  if (s->ev_rs_join) cudaEventDestroy(s->ev_rs_join);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

}  // namespace

extern "C" {

int32_t mithra_version(void) { return 100; }

const char* mithra_last_error(const mithra_sim* sim) {
  return sim ? sim->err.c_str() : g_thread_err.c_str();
}

mithra_status mithra_check_grid(const mithra_grid* grid) {
  std::string why;
  mithra_status st = check_grid(grid, &why);
  if (st != MITHRA_OK) return fail(nullptr, st, why);
  return MITHRA_OK;
}

mithra_status mithra_footprint(const mithra_grid* grid, int64_t n_particles,
                               mithra_precision precision, int64_t* bytes) {
  std::string why;
  mithra_status st = check_grid(grid, &why);
  if (st != MITHRA_OK) return fail(nullptr, st, why);
  if (!bytes || n_particles < 0) return fail(nullptr, MITHRA_EINVAL, "bad footprint arguments");
  int ntx, nty, ntz;
  tiles_of(grid, &ntx, &nty, &ntz);
  const int64_t nkeys = (int64_t)ntx * nty * ntz;
  const size_t r = real_size(precision);
  int64_t b = 4 * ncell_of(grid) * 4 * (int64_t)r;              // 2 levels, increment, sources
  if (has_lo(precision)) b += 2 * ncell_of(grid) * (int64_t)sizeof(LoV4);  // lo parts
  b += 2 * (int64_t)particle_buffer_bytes(n_particles, precision);
  b += 3 * n_particles * (int64_t)sizeof(int);                   // slot map, key, rank
  b += 3 * (nkeys + 2) * (int64_t)sizeof(int);                   // count, offset, tiles
  b += 8 * ((nkeys + 3) / 4);                                     // source-tile flags
  b += (nkeys / kScanBlock + 2) * (int64_t)sizeof(int4);         // scan block sums
  b += (int64_t)sizeof(StepState) + (int64_t)sizeof(double);
  *bytes = b;
  return MITHRA_OK;
}

mithra_status mithra_create(const mithra_grid* grid, const mithra_undulator* und,
                            const mithra_bunch* bunch, mithra_precision precision,
                            void* cuda_stream, mithra_sim** out) {
  if (!out) return fail(nullptr, MITHRA_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  mithra_status st = check_grid(grid, &why);
  if (st != MITHRA_OK) return fail(nullptr, st, why);
  if (!und) return fail(nullptr, MITHRA_EINVAL, "undulator is NULL");
  if (!(und->gamma0 > 1.0)) return fail(nullptr, MITHRA_EINVAL, "undulator needs gamma0 > 1");
  if (und->type == 1) {
    if (!(und->lambda_l > 0.0) || !(und->variance > 0.0) || !std::isfinite(und->a0) ||
        !(und->pol_x * und->pol_x + und->pol_y * und->pol_y > 0.0) ||
        (und->direction != 1 && und->direction != -1) || und->signal < 0 || und->signal > 3 ||
        !std::isfinite(und->offset) || !std::isfinite(und->z0_lab) || !std::isfinite(und->cep))
      return fail(nullptr, MITHRA_EINVAL,
                  "optical undulator needs lambda_l > 0, variance > 0, a polarization, "
                  "direction +-1 and signal 0..3");
    if (und->beam != 0)
      return fail(nullptr, MITHRA_EINVAL, "the optical undulator is a plane wave (beam 0)");
  } else if (und->type != 0 || !(und->lambda_u > 0.0)) {
    return fail(nullptr, MITHRA_EINVAL, "undulator type must be 0 (static, lambda_u > 0) or 1");
  }
  if (precision != MITHRA_P32 && precision != MITHRA_P64 && precision != MITHRA_P32_U64 &&
      precision != MITHRA_P32_C)
    return fail(nullptr, MITHRA_EINVAL,
                "precision must be MITHRA_P64, MITHRA_P32, MITHRA_P32_U64 or MITHRA_P32_C");
  const int64_t np = bunch ? bunch->n : 0;
  if (np < 0 || np >= ((int64_t)1 << 31)) return fail(nullptr, MITHRA_EINVAL, "bad particle count");
  if (np > 0 && (!bunch->x || !bunch->y || !bunch->z || !bunch->ux || !bunch->uy || !bunch->uz))
    return fail(nullptr, MITHRA_EINVAL, "bunch arrays must not be NULL");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
    return fail(nullptr, MITHRA_ENODEV, "no CUDA device");
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major != 10 || prop.minor != 3)
    return fail(nullptr, MITHRA_ENODEV, "this library is built for sm_103a (GB300) only");

  mithra_sim* s = new (std::nothrow) mithra_sim();
  if (!s) return fail(nullptr, MITHRA_ENOMEM, "host allocation failed");
  s->g = *grid;
  s->u = *und;
  s->prec = precision;
  s->q_macro = bunch ? bunch->q_macro : 0.0;
  s->np = np;
  tiles_of(grid, &s->ntx, &s->nty, &s->ntz);
  s->nkeys = s->ntx * s->nty * s->ntz;
  s->dirty_words = (s->nkeys + 3) / 4;
  auto bail = [&](mithra_status code, const std::string& msg) {
    free_all(s);
    delete s;
    return fail(nullptr, code, msg);
  };
  if (cuda_stream) {
    s->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(MITHRA_ECUDA, "stream creation failed");
    s->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_rs_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_rs_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(MITHRA_ECUDA, "side stream creation failed");
  const size_t r = real_size(precision);
  const size_t field_bytes = (size_t)ncell_of(grid) * 4 * r;
  auto dalloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes < 256 ? 256 : bytes) == cudaSuccess; };
  bool ok = dalloc(&s->P[0], field_bytes) && dalloc(&s->P[1], field_bytes) &&
            dalloc(&s->D, field_bytes) && dalloc(&s->S, field_bytes) &&
            dalloc(&s->pbuf[0], particle_buffer_bytes(np, precision)) &&
            dalloc(&s->pbuf[1], particle_buffer_bytes(np, precision)) &&
            dalloc((void**)&s->perm, sizeof(int) * (size_t)(np + 1)) &&
            dalloc((void**)&s->key, sizeof(int) * (size_t)(np + 1)) &&
            dalloc((void**)&s->rank, sizeof(int) * (size_t)(np + 1)) &&
            dalloc((void**)&s->count, sizeof(int) * (size_t)(s->nkeys + 2)) &&
            dalloc((void**)&s->offset, sizeof(int) * (size_t)(s->nkeys + 2)) &&
            dalloc((void**)&s->tiles, sizeof(int) * (size_t)(s->nkeys + 1)) &&
            dalloc((void**)&s->dirty, 8 * (size_t)s->dirty_words) &&
            dalloc((void**)&s->scan_part, sizeof(int4) * (size_t)(s->nkeys / kScanBlock + 2)) &&
            dalloc((void**)&s->dstate, sizeof(StepState)) &&
            dalloc((void**)&s->d_scalar, sizeof(double));
  const size_t lo_bytes = (size_t)ncell_of(grid) * sizeof(LoV4);
  if (ok && has_lo(precision))
    ok = dalloc(&s->PL[0], lo_bytes) && dalloc(&s->PL[1], lo_bytes);
  if (!ok) return bail(MITHRA_ENOMEM, "device allocation failed");
  if (cudaMallocHost((void**)&s->h_mirror, sizeof(*s->h_mirror)) != cudaSuccess)
    return bail(MITHRA_ENOMEM, "pinned allocation failed");
  s->h_mirror->n_lost = 0;
  s->h_mirror->err = 0;
  cudaMemsetAsync(s->P[0], 0, field_bytes, s->stream);
  cudaMemsetAsync(s->P[1], 0, field_bytes, s->stream);
  for (void* l : s->PL)
    if (l) cudaMemsetAsync(l, 0, lo_bytes, s->stream);
  cudaMemsetAsync(s->D, 0, field_bytes, s->stream);
  cudaMemsetAsync(s->S, 0, field_bytes, s->stream);
  cudaMemsetAsync(s->count, 0, sizeof(int) * (size_t)(s->nkeys + 2), s->stream);
  cudaMemsetAsync(s->dstate, 0, sizeof(StepState), s->stream);
  cudaMemsetAsync(s->dirty, 0, 8 * (size_t)s->dirty_words, s->stream);
  mark_sources_everywhere(s);
  {
    const int es = (int)r;
    s->have_tm = encode_field_map(&s->tm[0], s->P[0], es, grid->nx, grid->ny, grid->nz,
                                  kMX + 2, kMY + 2) &&
                 encode_field_map(&s->tm[1], s->P[1], es, grid->nx, grid->ny, grid->nz,
                                  kMX + 2, kMY + 2);
    s->have_tm = s->have_tm &&
                 encode_field_map(&s->tm_box[0], s->P[0], es, grid->nx, grid->ny, grid->nz, kTP,
                                  kTP, kTP) &&
                 encode_field_map(&s->tm_box[1], s->P[1], es, grid->nx, grid->ny, grid->nz, kTP,
                                  kTP, kTP) &&
                 encode_field_map(&s->tm_box_d, s->D, es, grid->nx, grid->ny, grid->nz, kTP, kTP,
                                  kTP) &&
                 encode_field_map(&s->tm_col_d, s->D, es, grid->nx, grid->ny, grid->nz, kMX, kMY) &&
                 encode_field_map(&s->tm_col_s, s->S, es, grid->nx, grid->ny, grid->nz, kMX, kMY);
    // defaults: the register z-marching update (fastest on every grid the
    // autotuner has timed, any precision) and the tiled push when TMA maps
    // exist
    s->stencil_variant = 2;
    s->push_variant = s->have_tm ? 1 : 0;
    st = with_types(precision, [&](auto t, auto u) {
      TYPES_OF(t, u);
      mithra_status r = setup_push_grid<T, U>(s);
      return r == MITHRA_OK ? setup_march<T>(s) : r;
    });
    s->lz = 16;
    if (st != MITHRA_OK) {
      std::string msg = s->err;
      return bail(st, msg);
    }
  }
  if (np > 0) {
    st = with_types(precision, [&](auto t, auto u) {
      TYPES_OF(t, u);
      return init_particles<T, U>(s, bunch);
    });
    if (st != MITHRA_OK) {
      std::string msg = s->err;
      return bail(st, msg);
    }
  }
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return bail(MITHRA_ECUDA, "set-up failed");
  *out = s;
  return MITHRA_OK;
}

namespace {
// Steps per captured graph of mithra_step (even).
constexpr int kGraphSteps = 4;

// Drops the captured steps of s (and of the batch s belongs to: a launch
// parameter of s changed).
void drop_step_graphs(mithra_sim* s) {
  for (auto& e : s->step_exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  if (s->in_batch) batch_mark_dirty(s->in_batch);
}

// Captures kGraphSteps steps from the current state (an even number: they
// bring the level and particle buffers back to it) into
// s->step_exec[s->cur]; each step's re-sort but the last runs beside the
// next step's potential update.
mithra_status capture_step_run(mithra_sim* s) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(s, e, "begin capture of the step");
  mithra_status st = MITHRA_OK;
  for (int k = 0; k < kGraphSteps && st == MITHRA_OK; ++k)
    st = with_types(s->prec, [&](auto t, auto u) {
      TYPES_OF(t, u);
      return launch_step<T, U>(s, k + 1 < kGraphSteps);
    });
  s->resort_pending = false;
  e = cudaStreamEndCapture(s->stream, &graph);
  if (st != MITHRA_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "end capture of the step");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(s, e, "instantiate the step graph");
  s->step_exec[s->cur] = ex;
  return MITHRA_OK;
}

mithra_status launch_one_step(mithra_sim* s) {
  mithra_status st = with_types(s->prec, [&](auto t, auto u) {
    TYPES_OF(t, u);
    return launch_step<T, U>(s);
  });
  if (st == MITHRA_OK) s->n_issued += 1;
  return st;
}
}  // namespace

mithra_status mithra_step(mithra_sim* s, int64_t n) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (n < 0) return fail(s, MITHRA_EINVAL, "n must be >= 0");
  if (s->h_mirror->err & 1) return fail(s, MITHRA_ENUMERIC, "NaN or Inf in a power reduction");
  if (s->strict_lost && s->h_mirror->n_lost > s->lost_base)
    return fail(s, MITHRA_ELOST, std::to_string(s->h_mirror->n_lost - s->lost_base) +
                                     " particle(s) left the valid region (strict mode)");
  if (s->in_batch) return fail(s, MITHRA_EBUSY, "sim belongs to a batch: step it with mithra_batch_step");
  int64_t t = 0;
  // runs of steps replay a captured run (no profiling events inside; the
  // legacy and per-thread default streams cannot be captured)
  bool graph = n >= kGraphSteps && !s->profiling && s->stream != nullptr &&
               s->stream != reinterpret_cast<cudaStream_t>(1) &&
               s->stream != reinterpret_cast<cudaStream_t>(2);
  if (graph) {  // a stream the caller is capturing takes the launches themselves
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s->stream, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
      graph = false;
  }
  if (graph) {
    if (!s->step_exec[s->cur]) {
      mithra_status st = capture_step_run(s);
      if (st != MITHRA_OK) return st;
    }
    for (; t + kGraphSteps <= n; t += kGraphSteps) {
      cudaError_t e = cudaGraphLaunch(s->step_exec[s->cur], s->stream);
      if (e != cudaSuccess) return cuda_fail(s, e, "step graph launch");
      s->n_issued += kGraphSteps;
    }
  }
  for (; t < n; ++t) {
    mithra_status st = launch_one_step(s);
    if (st != MITHRA_OK) return st;
  }
  refresh_mirror(s);
  return MITHRA_OK;
}

mithra_status mithra_sync(mithra_sim* s) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  return sync_status(s, true);
}

mithra_status mithra_set_lost_policy(mithra_sim* s, int32_t strict) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  const bool was = s->strict_lost;
  s->strict_lost = false;
  mithra_status st = sync_status(s);
  if (st != MITHRA_OK) {
    s->strict_lost = was;
    return st;
  }
  StepState d;
  MCHECK(s, cudaMemcpy(&d, s->dstate, sizeof(d), cudaMemcpyDeviceToHost));
  s->h_mirror->n_lost = d.n_lost;
  s->lost_base = d.n_lost;
  s->strict_lost = strict != 0;
  return MITHRA_OK;
}

mithra_status mithra_time(const mithra_sim* s, int64_t* n_steps, double* t) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (n_steps) *n_steps = s->n_issued;
  if (t) *t = s->t0 + (double)s->n_issued * s->g.dt;
  return MITHRA_OK;
}

mithra_status mithra_copy_field(mithra_sim* s, int32_t field, double* out) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (!out || field < 0 || field > MITHRA_PHI_PREV) return fail(s, MITHRA_EINVAL, "bad field id or NULL out");
  return s->prec == MITHRA_P64 ? copy_field_impl<double>(s, field, out)
                               : copy_field_impl<float>(s, field, out);
}

mithra_status mithra_set_field(mithra_sim* s, int32_t field, const double* in) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  drop_step_graphs(s);
  if (!in || field < 0 || field > MITHRA_PHI_PREV) return fail(s, MITHRA_EINVAL, "bad field id or NULL in");
  return s->prec == MITHRA_P64 ? set_field_impl<double>(s, field, in)
                               : set_field_impl<float>(s, field, in);
}

mithra_status mithra_sample_fields(mithra_sim* s, uint32_t mask, const int32_t* ijk, int64_t npts,
                                   double* out) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (npts == 0) return MITHRA_OK;
  if (!ijk || !out || npts < 0 || mask == 0 || (mask >> 14))
    return fail(s, MITHRA_EINVAL, "bad sampling arguments");
  for (int64_t p = 0; p < npts; ++p) {
    const int i = ijk[3 * p], j = ijk[3 * p + 1], k = ijk[3 * p + 2];
    if (i < 0 || i >= s->g.nx || j < 0 || j >= s->g.ny || k < 0 || k >= s->g.nz)
      return fail(s, MITHRA_EINVAL, "sample point outside the grid");
  }
  return s->prec == MITHRA_P64 ? sample_impl<double>(s, mask, ijk, npts, out)
                               : sample_impl<float>(s, mask, ijk, npts, out);
}

mithra_status mithra_radiated_power(mithra_sim* s, int32_t k_plane, double* p_lab, double* t_lab,
                                    double* z_lab) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (k_plane < 1 || k_plane > s->g.nz - 2) return fail(s, MITHRA_EINVAL, "k_plane outside [1, nz-2]");
  double p = 0.0;
  mithra_status st = s->prec == MITHRA_P64 ? power_impl<double>(s, k_plane, &p)
                                           : power_impl<float>(s, k_plane, &p);
  if (st != MITHRA_OK) return st;
  const double t = s->t0 + ((double)s->n_issued - 0.5) * s->g.dt;
  double tl, zl;
  lab_of(s, k_plane, t, &tl, &zl);
  if (p_lab) *p_lab = p;
  if (t_lab) *t_lab = tl;
  if (z_lab) *z_lab = zl;
  return MITHRA_OK;
}

mithra_status mithra_set_power_sampling(mithra_sim* s, int32_t k_plane, int64_t capacity) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  drop_step_graphs(s);
  if (capacity < 0) return fail(s, MITHRA_EINVAL, "capacity must be >= 0");
  if (capacity > 0 && (k_plane < 1 || k_plane > s->g.nz - 2))
    return fail(s, MITHRA_EINVAL, "k_plane outside [1, nz-2]");
  MCHECK(s, cudaStreamSynchronize(s->stream));
  if (s->d_power_rec) {
    cudaFree(s->d_power_rec);
    s->d_power_rec = nullptr;
  }
  s->power_cap = 0;
  if (capacity == 0) return MITHRA_OK;
  if (cudaMalloc((void**)&s->d_power_rec, sizeof(double) * (size_t)capacity) != cudaSuccess)
    return fail(s, MITHRA_ENOMEM, "power record allocation failed");
  MCHECK(s, cudaMemset(s->d_power_rec, 0, sizeof(double) * (size_t)capacity));
  s->power_cap = capacity;
  s->power_plane = k_plane;
  s->power_first = s->n_issued;
  return MITHRA_OK;
}

mithra_status mithra_read_power(mithra_sim* s, double* out, int64_t max_records, int64_t* count) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  int64_t have = s->n_issued - s->power_first;
  if (s->power_cap == 0) have = 0;
  if (have > s->power_cap) have = s->power_cap;
  if (count) *count = have;
  const int64_t m = have < max_records ? have : max_records;
  if (m <= 0 || !out) return sync_status(s);
  std::vector<double> p((size_t)m);
  MCHECK(s, cudaMemcpyAsync(p.data(), s->d_power_rec, sizeof(double) * m, cudaMemcpyDeviceToHost,
                            s->stream));
  mithra_status st = sync_status(s);
  if (st != MITHRA_OK) return st;
  for (int64_t r = 0; r < m; ++r) {
    const double t = s->t0 + ((double)(s->power_first + r) + 0.5) * s->g.dt;
    out[3 * r] = p[(size_t)r];
    lab_of(s, s->power_plane, t, &out[3 * r + 1], &out[3 * r + 2]);
  }
  return MITHRA_OK;
}

mithra_status mithra_set_seed(mithra_sim* s, const mithra_undulator* w) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  drop_step_graphs(s);
  if (s->in_batch) return fail(s, MITHRA_EBUSY, "sim is stepped by a batch");
  if (!w) {
    s->seed = SeedP{};
    return MITHRA_OK;
  }
  if (w->type != 1 || !(w->lambda_l > 0.0) || !(w->variance > 0.0) || !std::isfinite(w->a0) ||
      !(w->pol_x * w->pol_x + w->pol_y * w->pol_y > 0.0) ||
      (w->direction != 1 && w->direction != -1) || w->signal < 0 || w->signal > 3 ||
      !std::isfinite(w->offset) || !std::isfinite(w->z0_lab) || !std::isfinite(w->cep))
    return fail(s, MITHRA_EINVAL,
                "seed needs type 1, lambda_l > 0, variance > 0, a polarization, direction +-1 "
                "and signal 0..3");
  if (w->beam != 0 &&
      (w->beam != 1 || !(w->w_par > 0.0) || !(w->w_perp > 0.0) || !std::isfinite(w->w_par) ||
       !std::isfinite(w->w_perp) || !std::isfinite(w->x0_lab) || !std::isfinite(w->y0_lab)))
    return fail(s, MITHRA_EINVAL,
                "seed beam must be 0 (plane wave) or 1 (Gaussian beam with finite waists > 0 "
                "and a finite focus)");
  if (s->g.nz < 8 || s->g.nx < 4 || s->g.ny < 4)
    return fail(s, MITHRA_EINVAL, "seeding needs nz >= 8 (planes 2 and 3 inside)");
  const double g0 = s->u.gamma0;  // the simulation's frame
  const double b0 = std::sqrt(1.0 - 1.0 / (g0 * g0));
  const double d = w->direction;
  const double pn = std::sqrt(w->pol_x * w->pol_x + w->pol_y * w->pol_y);
  const double A0 = w->a0 * kMe * kC / kQe;
  const double tv = w->variance / kC;
  SeedP q{};
  q.on = 1;
  q.signal = w->signal;
  q.ax = A0 * w->pol_x / pn;
  q.ay = A0 * w->pol_y / pn;
  q.w0 = 2.0 * kPi * kC / w->lambda_l;
  q.cep = w->cep;
  q.t0o = w->offset / kC;
  q.inv_tv = 1.0 / tv;
  q.env_a = 2.0 * std::log(2.0) / (tv * tv);
  q.tau_t = g0 * (1.0 - d * b0);
  q.tau_z = g0 * (b0 - d) / kC;
  q.tau_c = d * w->z0_lab / kC;
  q.z2 = s->g.z0 + 2.0 * s->g.dz;
  q.z3 = s->g.z0 + 3.0 * s->g.dz;
  q.t0 = s->t0;
  q.dt = s->g.dt;
  if (w->beam == 1) {
    q.beam = 1;
    q.px = w->pol_x / pn;
    q.py = w->pol_y / pn;
    q.xf = w->x0_lab;
    q.yf = w->y0_lab;
    q.zeta_t = d * g0 * b0 * kC;  // zeta = d (z' - z_focus), z' = g0 (z + b0 c t)
    q.zeta_z = d * g0;
    q.zeta_c = -d * w->z0_lab;
    const double zp = kPi * w->w_par * w->w_par / w->lambda_l;
    const double zq = kPi * w->w_perp * w->w_perp / w->lambda_l;
    q.zr_p = zp;
    q.zr_q = zq;
    q.inv_w2p = 1.0 / (w->w_par * w->w_par);
    q.inv_w2q = 1.0 / (w->w_perp * w->w_perp);
    q.gx0 = s->g.x0;
    q.gy0 = s->g.y0;
    q.gdx = s->g.dx;
    q.gdy = s->g.dy;
    // the coupling of a vertex to the other plane (NSFD terms of the update)
    const double cdt = kC * s->g.dt;
    const double rx2 = (cdt / s->g.dx) * (cdt / s->g.dx), ry2 = (cdt / s->g.dy) * (cdt / s->g.dy);
    double A = 0.0;
    if (s->g.stencil == 0) {
      const double qx = s->g.dz / s->g.dx, qy = s->g.dz / s->g.dy;
      A = 0.25 * (1.0 + 0.02 / (qx * qx + qy * qy));  // Eq. NSFDCoefficient
    }
    q.kxA = rx2 * A;
    q.kyA = ry2 * A;
    q.kz2 = (cdt / s->g.dz) * (cdt / s->g.dz);
  }
  MCHECK(s, cudaStreamSynchronize(s->stream));
  s->seed = q;
  return MITHRA_OK;
}

mithra_status mithra_bunch_stats(mithra_sim* s, double k_b, double* out) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (!out || !std::isfinite(k_b)) return fail(s, MITHRA_EINVAL, "out is NULL or k_b not finite");
  if (s->np == 0) {
    for (int a = 0; a < 14; ++a) out[a] = 0.0;
    return sync_status(s);
  }
  return with_types(s->prec, [&](auto t, auto u) {
    TYPES_OF(t, u);
    return bunch_stats_impl<T, U>(s, k_b, out);
  });
}

mithra_status mithra_set_bunch_sampling(mithra_sim* s, double k_b, int32_t every,
                                        int64_t capacity) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  drop_step_graphs(s);
  if (s->in_batch) return fail(s, MITHRA_EBUSY, "sim is stepped by a batch");
  if (every < 0 || capacity < 0 || !std::isfinite(k_b))
    return fail(s, MITHRA_EINVAL, "every and capacity must be >= 0, k_b finite");
  MCHECK(s, cudaStreamSynchronize(s->stream));
  if (s->d_bunch_rec) cudaFree(s->d_bunch_rec);
  if (s->d_bunch_part) cudaFree(s->d_bunch_part);
  s->d_bunch_rec = s->d_bunch_part = nullptr;
  s->bunch_every = 0;
  s->bunch_cap = 0;
  if (every == 0 || capacity == 0 || s->np == 0) return MITHRA_OK;
  if (cudaMalloc((void**)&s->d_bunch_rec, sizeof(double) * 15 * (size_t)capacity) != cudaSuccess ||
      cudaMalloc((void**)&s->d_bunch_part, sizeof(double) * 1024 * kBunchSums) != cudaSuccess)
    return fail(s, MITHRA_ENOMEM, "bunch record allocation failed");
  MCHECK(s, cudaMemset(s->d_bunch_rec, 0, sizeof(double) * 15 * (size_t)capacity));
  s->bunch_every = every;
  s->bunch_kb = k_b;
  s->bunch_first = s->n_issued;
  s->bunch_cap = capacity;
  return MITHRA_OK;
}

mithra_status mithra_read_bunch(mithra_sim* s, double* out, int64_t max_records, int64_t* count) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  int64_t have = s->bunch_every > 0 ? (s->n_issued - s->bunch_first) / s->bunch_every : 0;
  if (have > s->bunch_cap) have = s->bunch_cap;
  if (count) *count = have;
  const int64_t m = have < max_records ? have : max_records;
  if (m <= 0 || !out) return sync_status(s);
  MCHECK(s, cudaMemcpyAsync(out, s->d_bunch_rec, sizeof(double) * 15 * (size_t)m,
                            cudaMemcpyDeviceToHost, s->stream));
  return sync_status(s);
}

mithra_status mithra_set_spectrum(mithra_sim* s, int32_t k_plane, int32_t n_wavelengths,
                                  const double* lambda_lab) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  drop_step_graphs(s);
  if (s->in_batch) return fail(s, MITHRA_EBUSY, "sim is stepped by a batch");
  if (n_wavelengths < 0 || n_wavelengths > kMaxSpectrum)
    return fail(s, MITHRA_EINVAL, "n_wavelengths outside [0, 64]");
  if (n_wavelengths > 0) {
    if (k_plane < 1 || k_plane > s->g.nz - 2)
      return fail(s, MITHRA_EINVAL, "k_plane outside [1, nz-2]");
    if (!lambda_lab) return fail(s, MITHRA_EINVAL, "lambda_lab is NULL");
    for (int m = 0; m < n_wavelengths; ++m)
      if (!(lambda_lab[m] > 0.0) || !std::isfinite(lambda_lab[m]))
        return fail(s, MITHRA_EINVAL, "wavelengths must be finite and > 0");
  }
  MCHECK(s, cudaStreamSynchronize(s->stream));
  free_spectrum(s);
  if (n_wavelengths == 0) return MITHRA_OK;
  const long long nv = (long long)(s->g.nx - 2) * (s->g.ny - 2);
  const size_t acc_bytes = sizeof(double) * 8 * (size_t)nv * (size_t)n_wavelengths;
  if (cudaMalloc((void**)&s->d_spec_omega, sizeof(double) * n_wavelengths) != cudaSuccess ||
      cudaMalloc((void**)&s->d_spec_acc, acc_bytes) != cudaSuccess ||
      cudaMalloc((void**)&s->d_spec_out, sizeof(double) * n_wavelengths) != cudaSuccess ||
      cudaMalloc((void**)&s->d_spec_samples, sizeof(long long)) != cudaSuccess) {
    free_spectrum(s);
    return fail(s, MITHRA_ENOMEM, "spectrum allocation failed");
  }
  // a forward lab wave of wavelength lambda passes the plane, which moves
  // with the rest frame at beta0 c, at angular frequency 2 pi c (1 - beta0) / lambda
  const double g0 = s->u.gamma0;
  const double b0 = std::sqrt(1.0 - 1.0 / (g0 * g0));
  std::vector<double> om((size_t)n_wavelengths);
  for (int m = 0; m < n_wavelengths; ++m) om[m] = 2.0 * kPi * kC * (1.0 - b0) / lambda_lab[m];
  MCHECK(s, cudaMemcpy(s->d_spec_omega, om.data(), sizeof(double) * n_wavelengths,
                       cudaMemcpyHostToDevice));
  MCHECK(s, cudaMemset(s->d_spec_acc, 0, acc_bytes));
  MCHECK(s, cudaMemset(s->d_spec_samples, 0, sizeof(long long)));
  s->spec_plane = k_plane;
  s->spec_nf = n_wavelengths;
  return MITHRA_OK;
}

mithra_status mithra_read_spectrum(mithra_sim* s, double* dW_domega, int64_t* n_samples) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (s->spec_nf == 0) {
    if (n_samples) *n_samples = 0;
    return sync_status(s);
  }
  const long long nv = (long long)(s->g.nx - 2) * (s->g.ny - 2);
  k_spectrum_density<<<s->spec_nf, 256, 0, s->stream>>>(s->d_spec_acc, nv,
                                                        s->g.dx * s->g.dy / (kPi * kMu0),
                                                        s->d_spec_out);
  MCHECK(s, cudaGetLastError());
  long long ns = 0;
  if (dW_domega)
    MCHECK(s, cudaMemcpyAsync(dW_domega, s->d_spec_out, sizeof(double) * s->spec_nf,
                              cudaMemcpyDeviceToHost, s->stream));
  MCHECK(s, cudaMemcpyAsync(&ns, s->d_spec_samples, sizeof(long long), cudaMemcpyDeviceToHost,
                            s->stream));
  mithra_status st = sync_status(s);
  if (n_samples) *n_samples = ns;
  return st;
}

mithra_status mithra_copy_particles(mithra_sim* s, double* x, double* y, double* z, double* ux,
                                    double* uy, double* uz, int32_t* lost, int64_t* n_lost) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (s->np > 0 && (x || y || z || ux || uy || uz || lost)) {
    std::vector<double> buf((size_t)s->np * 7);
    mithra_status st = with_types(s->prec, [&](auto t, auto u) {
      TYPES_OF(t, u);
      return copy_particles_impl<T, U>(s, buf.data());
    });
    if (st != MITHRA_OK) return st;
    double* dst[6] = {x, y, z, ux, uy, uz};
    for (int a = 0; a < 6; ++a)
      if (dst[a]) std::memcpy(dst[a], buf.data() + (size_t)a * s->np, sizeof(double) * s->np);
    if (lost)
      for (int64_t q = 0; q < s->np; ++q) lost[q] = buf[(size_t)6 * s->np + q] != 0.0 ? 1 : 0;
  }
  if (n_lost) {
    StepState st;
    MCHECK(s, cudaStreamSynchronize(s->stream));
    MCHECK(s, cudaMemcpy(&st, s->dstate, sizeof(st), cudaMemcpyDeviceToHost));
    *n_lost = st.n_lost;
  }
  return MITHRA_OK;
}

mithra_status mithra_profile(mithra_sim* s, int32_t enable) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (enable && !s->profiling) {
    for (int k = 0; k < K_COUNT; ++k) { s->prof_ms[k] = 0.0; s->prof_n[k] = 0; }
  }
  s->profiling = enable != 0;
  return MITHRA_OK;
}

mithra_status mithra_kernel_times(mithra_sim* s, double* ms, int64_t* launches,
                                  int32_t max_kernels, int32_t* n_kernels) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  MCHECK(s, cudaStreamSynchronize(s->stream));
  flush_profile(s);
  if (n_kernels) *n_kernels = K_COUNT;
  for (int k = 0; k < K_COUNT && k < max_kernels; ++k) {
    if (ms) ms[k] = s->prof_ms[k];
    if (launches) launches[k] = s->prof_n[k];
  }
  return MITHRA_OK;
}

mithra_status mithra_source_tiles(mithra_sim* s, int64_t* marked, int32_t* everywhere) {
  if (!s || !marked || !everywhere) return fail(s, MITHRA_EINVAL, "sim and outputs must not be NULL");
  std::vector<unsigned char> f((size_t)4 * s->dirty_words);
  int all = 0;
  MCHECK(s, cudaMemcpyAsync(f.data(), s->dirty + (size_t)s->cur * 4 * s->dirty_words, f.size(),
                            cudaMemcpyDeviceToHost, s->stream));
  MCHECK(s, cudaMemcpyAsync(&all, &s->dstate->src_all[s->cur], sizeof(int),
                            cudaMemcpyDeviceToHost, s->stream));
  MCHECK(s, cudaStreamSynchronize(s->stream));
  int64_t n = 0;
  for (int t = 0; t < s->nkeys; ++t) n += f[t] != 0;
  *marked = n;
  *everywhere = all != 0;
  return MITHRA_OK;
}

const char* mithra_kernel_name(int32_t kernel) {
  return (kernel >= 0 && kernel < K_COUNT) ? kKernelNames[kernel] : nullptr;
}

mithra_status mithra_set_tuning(mithra_sim* s, const mithra_tuning* t) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  drop_step_graphs(s);
  if (!t || t->stencil_variant < 0 || t->stencil_variant > 2 || t->lz < 0 ||
      t->push_variant < 0 || t->push_variant > 1 || t->push_ctas_per_sm < 0 ||
      t->push_sparse_below < 0)
    return fail(s, MITHRA_EINVAL,
                "bad tuning: stencil variant 0..2, push variant 0 or 1, lz >= 0, ctas >= 0, "
                "sparse_below >= 0");
  if ((t->stencil_variant == 1 || t->push_variant == 1) && !s->have_tm)
    return fail(s, MITHRA_EINVAL, "TMA tensor maps unavailable: variant 1 disabled");
  if (t->stencil_variant == 1 && s->PL[0])
    return fail(s, MITHRA_EINVAL,
                "the marching update keeps single-float levels: not with compensated levels");
  s->stencil_variant = t->stencil_variant;
  s->lz = t->lz > 0 ? t->lz : (t->stencil_variant == 2 ? 16 : default_lz(&s->g, s->march_resident));
  s->push_variant = t->push_variant;
  s->push_ctas_per_sm = t->push_ctas_per_sm;
  s->push_sparse_below = t->push_sparse_below;
  const int per_sm = (t->push_ctas_per_sm > 0 && t->push_ctas_per_sm < s->push_max_per_sm)
                         ? t->push_ctas_per_sm
                         : s->push_max_per_sm;
  s->push_grid = s->n_sm * per_sm;
  return MITHRA_OK;
}

mithra_status mithra_get_tuning(const mithra_sim* s, mithra_tuning* t) {
  if (!s) return fail(nullptr, MITHRA_EINVAL, "sim is NULL");
  if (!t) return fail(nullptr, MITHRA_EINVAL, "tuning is NULL");
  t->stencil_variant = s->stencil_variant;
  t->lz = s->lz;
  t->push_variant = s->push_variant;
  t->push_ctas_per_sm = s->push_ctas_per_sm;
  t->push_sparse_below = s->push_sparse_below;
  return MITHRA_OK;
}

// ---- snapshot and restore -------------------------------------------------
// The device state a later step reads: both potential levels (and their lo
// parts), the increment, the sources, the particle buffer in use, the tile
// counts, offsets and list of the last re-sort, and the step state (device
// clock, lost count, error word); after a header that identifies the
// simulation's shape.
namespace {

constexpr uint64_t kSnapMagic = 0x31504e5348544d4dULL;

struct SnapHeader {
  uint64_t magic;
  int32_t prec, nx, ny, nz, nkeys, has_lo, cur, pb;
  int64_t np, n_issued;
  double t0;
};

struct SnapPart {
  void* dev;
  size_t bytes;
};

std::vector<SnapPart> snap_parts(const mithra_sim* s) {
  const size_t cells = (size_t)ncell_of(&s->g);
  const size_t fb = cells * 4 * real_size(s->prec);
  std::vector<SnapPart> v = {{s->P[0], fb}, {s->P[1], fb}, {s->D, fb}, {s->S, fb}};
  if (s->PL[0]) {
    v.push_back({s->PL[0], cells * sizeof(LoV4)});
    v.push_back({s->PL[1], cells * sizeof(LoV4)});
  }
  v.push_back({s->pbuf[s->pb], particle_buffer_bytes(s->np, s->prec)});
  v.push_back({s->perm, sizeof(int) * (size_t)s->np});
  v.push_back({s->count, sizeof(int) * (size_t)(s->nkeys + 2)});
  v.push_back({s->offset, sizeof(int) * (size_t)(s->nkeys + 2)});
  v.push_back({s->tiles, sizeof(int) * (size_t)(s->nkeys + 1)});
  v.push_back({s->dstate, sizeof(StepState)});
  return v;
}

}  // namespace

mithra_status mithra_snapshot_bytes(const mithra_sim* s, int64_t* bytes) {
  if (!s || !bytes) return fail(nullptr, MITHRA_EINVAL, "sim or bytes is NULL");
  int64_t b = sizeof(SnapHeader);
  for (const SnapPart& part : snap_parts(s)) b += (int64_t)part.bytes;
  *bytes = b;
  return MITHRA_OK;
}

mithra_status mithra_snapshot(mithra_sim* s, void* out) {
  if (!s || !out) return fail(s, MITHRA_EINVAL, "sim or out is NULL");
  mithra_status st = sync_status(s);
  if (st != MITHRA_OK) return st;
  SnapHeader h{kSnapMagic, s->prec, s->g.nx, s->g.ny, s->g.nz, s->nkeys, s->PL[0] ? 1 : 0,
               s->cur, s->pb, s->np, s->n_issued, s->t0};
  unsigned char* o = static_cast<unsigned char*>(out);
  std::memcpy(o, &h, sizeof(h));
  size_t at = sizeof(h);
  for (const SnapPart& part : snap_parts(s)) {
    MCHECK(s, cudaMemcpyAsync(o + at, part.dev, part.bytes, cudaMemcpyDeviceToHost, s->stream));
    at += part.bytes;
  }
  return sync_status(s);
}

mithra_status mithra_restore(mithra_sim* s, const void* in) {
  if (!s || !in) return fail(s, MITHRA_EINVAL, "sim or in is NULL");
  if (s->in_batch) return fail(s, MITHRA_EBUSY, "sim is stepped by a batch");
  SnapHeader h;
  std::memcpy(&h, in, sizeof(h));
  if (h.magic != kSnapMagic || h.prec != s->prec || h.nx != s->g.nx || h.ny != s->g.ny ||
      h.nz != s->g.nz || h.nkeys != s->nkeys || h.has_lo != (s->PL[0] ? 1 : 0) ||
      h.np != s->np || (h.cur & ~1) != 0 || (h.pb & ~1) != 0)
    return fail(s, MITHRA_EINVAL, "snapshot of another grid, precision or particle count");
  MCHECK(s, cudaStreamSynchronize(s->stream));
  drop_step_graphs(s);
  s->cur = h.cur;
  s->pb = h.pb;
  s->n_issued = h.n_issued;
  s->t0 = h.t0;
  // the diagnostics' records are not part of the state: restoring stops them
  s->power_cap = 0;
  s->bunch_every = 0;
  s->spec_nf = 0;
  const unsigned char* p = static_cast<const unsigned char*>(in) + sizeof(h);
  for (const SnapPart& part : snap_parts(s)) {
    MCHECK(s, cudaMemcpyAsync(part.dev, p, part.bytes, cudaMemcpyHostToDevice, s->stream));
    p += part.bytes;
  }
  mark_sources_everywhere(s);
  MCHECK(s, refresh_mirror(s));
  mithra_status st = sync_status(s);
  // a strict count starts again from the restored state
  if (s->strict_lost) s->lost_base = s->h_mirror->n_lost;
  return st;
}

mithra_status mithra_boost_from_lab(const mithra_lab_case* lab, mithra_rest_frame* out) {
  if (!lab || !out) return fail(nullptr, MITHRA_EINVAL, "lab or out is NULL");
  if (!(lab->gamma > 1.0) || !(lab->lambda_u > 0.0) || !(lab->K >= 0.0) ||
      lab->steps_per_period < 1 || !(lab->courant > 0.0 && lab->courant <= 1.0) ||
      !(lab->sigma_gamma_rel >= 0.0))
    return fail(nullptr, MITHRA_EINVAL, "bad lab case");
  const double g = lab->gamma;
  const double g0 = g / std::sqrt(1.0 + 0.5 * lab->K * lab->K);
  const double b0 = std::sqrt(1.0 - 1.0 / (g0 * g0));
  const double b = std::sqrt(1.0 - 1.0 / (g * g));
  const double shift = g0 * (1.0 - b * b0);  // gamma_rest / gamma of the beam
  const double gr = g * shift;
  const double cdt = lab->lambda_u / g0 / lab->steps_per_period;
  out->gamma0 = g0;
  out->beta0 = b0;
  out->dt = cdt / kC;
  out->dz = cdt / lab->courant;
  out->uz_mean = std::sqrt(std::max(gr * gr - 1.0, 0.0));
  out->uz_sigma = g * lab->sigma_gamma_rel * shift;
  out->k_b = g0 * 2.0 * kPi / lab->lambda_u * (1.0 + b0);
  out->lambda_r_lab = lab->lambda_u * (1.0 + 0.5 * lab->K * lab->K) / (2.0 * g * g);
  return MITHRA_OK;
}

mithra_status mithra_destroy(mithra_sim* s) {
  if (!s) return MITHRA_OK;
  if (s->in_batch) mithra_batch_remove(s->in_batch, s);
  free_all(s);
  delete s;
  return MITHRA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched stepping: one CUDA graph advances every member by two steps.  Each
// member's kernels stay on its own stream; the graph forks from the batch's
// stream to every member stream and joins back, so independent members run
// concurrently.  Two steps bring each member's ping-pong buffers back to the
// state they had at capture, so the same graph serves every later pair of
// steps; it is captured again only when the membership changes.

struct mithra_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<mithra_sim*> sims;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
  cudaEvent_t fork = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> joins;
  std::string err;
  // fused form (batch_kernels.cuh): one launch per phase over all members
  int mode = 2;           // mithra_batch_set_mode: 0 per member, 1 fused, 2 automatic
  bool fused_now = false;  // the captured graph is the fused form
  void* d_table = nullptr;  // member tables of the two captured steps
  size_t table_bytes = 0;
  int* d_blk = nullptr;     // block prefixes, kBPCount x (M + 1)
  size_t blk_bytes = 0;
  int* d_pref = nullptr;    // the particle step's tile prefix (M + 1) and counter
  size_t pref_bytes = 0;
  int* d_zblk = nullptr;    // boundary and update block prefixes, per group from 0
  size_t zblk_bytes = 0;
  int push_grid = 0;
  // captures so far, their host time, and how many were fused
  int64_t captures = 0, fused_captures = 0;
  double capture_s = 0.0;
};

void batch_mark_dirty(mithra_batch* b) {
  if (b) b->dirty = true;
}

namespace {

mithra_status bfail(mithra_batch* b, mithra_status st, const std::string& msg) {
  if (b) b->err = msg; else g_thread_err = msg;
  return st;
}

void drop_graph(mithra_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->dirty = true;
}

// Whether every member can take the fused form: one precision form and
// undulator type, the register z-marching update, the tiled particle step
// with its tensor maps, and none of the per-step extras the batched kernels
// leave out (seed, spectrum, bunch recording).
// Average work of a member in cell-update equivalents (a particle step costs
// about four cell updates on GB300), the automatic mode's measure of size.
double member_work(const mithra_batch* b) {
  double w = 0.0;
  for (const mithra_sim* s : b->sims)
    w += (double)ncell_of(&s->g) + 4.0 * (double)s->np * s->g.n_sub;
  return w / (double)b->sims.size();
}

// Below this average member size the fused form is faster (measured on
// GB300: 64 and 256 members of 32 x 32 x 128 cells and 2000 particles ran
// 1.3x and 3.8x faster fused; members of 0.3 M cells and 0.2 M particles, and
// the c4 design sweep of 4 M cells and 2.3 M particles per member, ran 5 %
// and 2 % faster as one launch sequence per member, whose members' phases
// overlap on the device).
constexpr double kFuseBelowWork = 5.0e5;

bool fusable(const mithra_batch* b) {
  if (b->mode == 0 || b->sims.empty()) return false;
  if (b->mode == 2 && member_work(b) >= kFuseBelowWork) return false;
  const mithra_sim* f = b->sims[0];
  for (const mithra_sim* s : b->sims) {
    if (s->prec != f->prec || s->u.type != f->u.type || s->g.boundary != f->g.boundary)
      return false;
    if (s->stencil_variant != 2 || s->push_variant != 1 || !s->have_tm) return false;
    if (s->seed.on || s->spec_nf > 0 || s->bunch_every > 0) return false;
  }
  return true;
}

mithra_status grow(mithra_batch* b, void** p, size_t* have, size_t need) {
  if (*have >= need) return MITHRA_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) return bfail(b, MITHRA_ENOMEM, "batch table allocation");
  *have = need;
  return MITHRA_OK;
}

// Member table entry of s for the step that starts with level buffer c and
// particle buffer pb.
template <typename T, typename U>
BatchMember<T, U> member_entry(mithra_sim* s, int c, int pb) {
  BatchMember<T, U> m{};
  m.sp = make_stencil<T>(s->g);
  m.pp = make_pic<T>(s);
  m.P0 = static_cast<V4<T>*>(s->P[c]);
  m.P1 = static_cast<V4<T>*>(s->P[1 - c]);
  m.L0 = static_cast<LoV4*>(s->PL[c]);
  m.L1 = static_cast<LoV4*>(s->PL[1 - c]);
  m.pp.plo = m.L1;
  m.D = static_cast<V4<T>*>(s->D);
  m.S = static_cast<V4<T>*>(s->S);
  m.A = parts_of<T, U>(s, pb);
  m.B = parts_of<T, U>(s, 1 - pb);
  m.perm = s->perm;
  m.offset = s->offset;
  m.tiles = s->tiles;
  m.count = s->count;
  m.key = s->key;
  m.rank = s->rank;
  m.scan_part = s->scan_part;
  m.st = s->dstate;
  m.power_acc = s->d_power_rec ? s->d_power_rec - s->power_first : nullptr;
  m.power_end = s->power_cap > 0 ? s->power_first + s->power_cap : 0;
  m.g0 = s->u.gamma0;
  m.b0 = std::sqrt(1.0 - 1.0 / (s->u.gamma0 * s->u.gamma0));
  m.np = s->np;
  m.lz = s->lz;
  m.power_plane = s->power_plane;
  m.nkeys = s->nkeys;
  m.scan_nb = (s->nkeys + 1 + kScanBlock - 1) / kScanBlock;
  m.sparse_below = 0;  // the fused particle step stages every tile
  m.fused_mur = s->g.boundary == 1;
  set_source_flags(s, c, &m.sp);
  m.dirty = s->dirty;
  m.dirty_words = s->dirty_words;
  m.cur = c;
  return m;
}

// The particle step's arguments of a member table entry.
template <typename T, typename U>
PushArgs<T, U> push_args_of(const BatchMember<T, U>& m) {
  PushArgs<T, U> a;
  a.p = m.pp;
  a.st = m.st;
  a.pn = m.P1;
  a.D = m.D;
  a.src = m.S;
  a.P = m.A;
  a.O = m.B;
  a.perm = m.perm;
  a.offset = m.offset;
  a.tiles = m.tiles;
  a.count = m.count;
  a.key = m.key;
  a.rank = m.rank;
  a.lost_ctr = &m.st->n_lost;
  a.np = m.np;
  a.dirty = m.dirty;
  a.dirty_words = m.dirty_words;
  a.cur = m.cur;
  return a;
}

template <typename T, typename U>
mithra_status capture_fused_typed(mithra_batch* b) {
  const int M = (int)b->sims.size();
  std::vector<BatchMember<T, U>> tab(2 * (size_t)M);
  std::vector<BatchMaps> maps(2 * (size_t)M);
  std::vector<int> blk((size_t)kBPCount * (M + 1), 0);
  for (int k = 0; k < M; ++k) {
    mithra_sim* s = b->sims[k];
    for (int t = 0; t < 2; ++t) {
      const int c = t == 0 ? s->cur : 1 - s->cur;
      const int pb = t == 0 ? s->pb : 1 - s->pb;
      tab[(size_t)t * M + k] = member_entry<T, U>(s, c, pb);
      maps[(size_t)t * M + k].box = s->tm_box[1 - c];
      maps[(size_t)t * M + k].box_d = s->tm_box_d;
    }
    const mithra_grid& g = s->g;
    const long long nb[kBPCount] = {
        (long long)blocks_for(batch_mur_count(g.nx, g.ny, g.nz, g.boundary == 1), 256),
        (long long)((g.nx + 31) / 32) * ((g.ny + 7) / 8) * ((g.nz + s->lz - 1) / s->lz),
        s->power_cap > 0 ? kBatchPowerBlocks : 0,
        (long long)((s->nkeys + 1 + kScanBlock - 1) / kScanBlock),
        s->np > 0 ? (long long)blocks_for(s->np, 256) : 0};
    for (int ph = 0; ph < kBPCount; ++ph) {
      const long long v = blk[(size_t)ph * (M + 1) + k] + nb[ph];
      if (v >= (1LL << 31)) return bfail(b, MITHRA_EINVAL, "batch work list exceeds 2^31 blocks");
      blk[(size_t)ph * (M + 1) + k + 1] = (int)v;
    }
  }
  mithra_status st = grow(b, &b->d_table, &b->table_bytes, sizeof(BatchMember<T, U>) * tab.size());
  if (st == MITHRA_OK)
    st = grow(b, reinterpret_cast<void**>(&b->d_blk), &b->blk_bytes, sizeof(int) * blk.size());
  const int npg = (M + kPushGroup - 1) / kPushGroup;
  if (st == MITHRA_OK)
    st = grow(b, reinterpret_cast<void**>(&b->d_pref), &b->pref_bytes,
              sizeof(int) * (size_t)(M + 2 * npg));
  // block prefixes of the boundary and update phases, restarted at 0 for
  // each group of kZGroup members (M + 1 per group's entries)
  const int ngroups = (M + kZGroup - 1) / kZGroup;
  std::vector<int> zblk(2 * (size_t)(M + ngroups), 0);
  for (int pi = 0; pi < 2; ++pi) {
    const int ph = pi == 0 ? kBPMur : kBPZ;
    for (int g0 = 0; g0 < M; g0 += kZGroup) {
      const int Mg = std::min(kZGroup, M - g0);
      int* z = zblk.data() + (size_t)pi * (M + ngroups) + g0 + g0 / kZGroup;
      for (int k = 0; k <= Mg; ++k) z[k] = blk[(size_t)ph * (M + 1) + g0 + k] - blk[(size_t)ph * (M + 1) + g0];
    }
  }
  if (st == MITHRA_OK)
    st = grow(b, reinterpret_cast<void**>(&b->d_zblk), &b->zblk_bytes, sizeof(int) * zblk.size());
  if (st != MITHRA_OK) return st;
  if (cudaMemcpy(b->d_zblk, zblk.data(), sizeof(int) * zblk.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return bfail(b, MITHRA_ECUDA, "batch table upload");
  // the tables replace the ones the previous graph read: after its work
  if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
      cudaMemcpy(b->d_table, tab.data(), sizeof(BatchMember<T, U>) * tab.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_blk, blk.data(), sizeof(int) * blk.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return bfail(b, MITHRA_ECUDA, "batch table upload");
  const bool opt = b->sims[0]->u.type == 1;
  const bool lo = b->sims[0]->PL[0] != nullptr;
  constexpr bool kAnyLo = sizeof(T) == 4;  // compensated levels exist for FP32 fields only
  const int smem = tile_smem_bytes<T, U>();
  auto kpush = opt ? (lo ? k_push_tiled<true, T, U, kAnyLo, true>
                        : k_push_tiled<true, T, U, false, true>)
                   : (lo ? k_push_tiled<false, T, U, kAnyLo, true>
                         : k_push_tiled<false, T, U, false, true>);
  if (cudaFuncSetAttribute(kpush, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return bfail(b, MITHRA_ECUDA, "batched particle step: shared memory attribute");
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kpush, kPushThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return bfail(b, MITHRA_ECUDA, "batched particle step does not fit an SM");
  b->push_grid = b->sims[0]->n_sm * per_sm;
  auto total = [&](int ph) { return blk[(size_t)ph * (M + 1) + M]; };
  const int* dblk = b->d_blk;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(b, MITHRA_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  for (int t = 0; t < 2; ++t) {
    const BatchMember<T, U>* mem = static_cast<const BatchMember<T, U>*>(b->d_table) + (size_t)t * M;
    cudaStream_t q = b->stream;
    // boundary and potential update, one launch each per group of up to
    // kZGroup members (their arguments in the launch's parameter space);
    // the groups' block numbers start at the group's first member
    for (int g0 = 0; g0 < M; g0 += kZGroup) {
      const int Mg = std::min(kZGroup, M - g0);
      ZParams<T> zp;
      for (int k = 0; k < Mg; ++k) {
        const BatchMember<T, U>& e = tab[(size_t)t * M + g0 + k];
        zp.m[k] = ZMember<T>{e.sp, e.P0, e.L0, e.P1, e.L1, e.D, e.S, e.lz, e.fused_mur};
      }
      zp.M = Mg;
      for (int ph : {(int)kBPMur, (int)kBPZ}) {
        const int* pb = blk.data() + (size_t)ph * (M + 1);
        const int nblk = pb[g0 + Mg] - pb[g0];
        if (nblk == 0) continue;
        zp.blk = b->d_zblk + (size_t)(ph == kBPMur ? 0 : 1) * (M + ngroups) + g0 + g0 / kZGroup;
        if (ph == kBPMur) {
          if (lo) kb_mur<kAnyLo, T><<<nblk, 256, 0, q>>>(zp);
          else kb_mur<false, T><<<nblk, 256, 0, q>>>(zp);
        } else if (b->sims[0]->g.boundary == 1) {
          if (lo) kb_potential<kAnyLo, T, true><<<nblk, dim3(32, 8), 0, q>>>(zp);
          else kb_potential<false, T, true><<<nblk, dim3(32, 8), 0, q>>>(zp);
        } else {
          if (lo) kb_potential<kAnyLo, T, false><<<nblk, dim3(32, 8), 0, q>>>(zp);
          else kb_potential<false, T, false><<<nblk, dim3(32, 8), 0, q>>>(zp);
        }
      }
    }
    if (total(kBPPow) > 0)
      kb_power<T, U><<<total(kBPPow), 256, 0, q>>>(mem, dblk + kBPPow * (M + 1), M);
    // the particle step, one launch per group of up to kPushGroup members
    // (their arguments in the launch's parameter space)
    for (int g0 = 0; g0 < M; g0 += kPushGroup) {
      const int Mg = std::min(kPushGroup, M - g0);
      int* pref = b->d_pref + g0 + 2 * (g0 / kPushGroup);  // Mg + 1 entries, then the counter
      int* work = pref + Mg + 1;
      kb_tile_prefix<T, U><<<1, 1024, 0, q>>>(mem + g0, Mg, pref, work);
      PushParams<T, U, true> prm;
      for (int k = 0; k < Mg; ++k) {
        prm.m[k] = push_args_of(tab[(size_t)t * M + g0 + k]);
        prm.box[k] = maps[(size_t)t * M + g0 + k].box;
        prm.box_d[k] = maps[(size_t)t * M + g0 + k].box_d;
      }
      prm.pref = pref;
      prm.work = work;
      prm.M = Mg;
      kpush<<<b->push_grid, kPushThreads, smem, q>>>(prm);
    }
    kb_scan_partials<T, U><<<total(kBPScan), kScanBlock, 0, q>>>(mem, dblk + kBPScan * (M + 1), M);
    kb_scan_final<T, U><<<total(kBPScan), kScanBlock, 0, q>>>(mem, dblk + kBPScan * (M + 1), M);
    if (total(kBPSlot) > 0)
      kb_slot_map<T, U><<<total(kBPSlot), 256, 0, q>>>(mem, dblk + kBPSlot * (M + 1), M);
  }
  cudaError_t le = cudaGetLastError();
  e = cudaStreamEndCapture(b->stream, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, MITHRA_ECUDA, std::string("batched launch: ") + cudaGetErrorString(le));
  }
  if (e != cudaSuccess) return bfail(b, MITHRA_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, MITHRA_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  b->fused_now = true;
  b->dirty = false;
  return MITHRA_OK;
}

mithra_status capture_graph(mithra_batch* b);

// Captures the batch's two-step graph in the fused or the per-member form,
// counting the captures and their host time.
mithra_status capture(mithra_batch* b) {
  const auto t0 = std::chrono::steady_clock::now();
  // the graph launched last may still be reading the device tables that the
  // capture rewrites (with copies outside the batch's stream): let it finish
  const cudaError_t se = cudaStreamSynchronize(b->stream);
  if (se != cudaSuccess)
    return bfail(b, MITHRA_ECUDA, std::string("batch stream: ") + cudaGetErrorString(se));
  drop_graph(b);
  b->fused_now = false;
  mithra_status st;
  if (fusable(b))
    st = with_types(b->sims[0]->prec, [&](auto tt, auto uu) {
      TYPES_OF(tt, uu);
      return capture_fused_typed<T, U>(b);
    });
  else
    st = capture_graph(b);
  b->captures += 1;
  b->fused_captures += b->fused_now ? 1 : 0;
  b->capture_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

mithra_status capture_graph(mithra_batch* b) {
  while (b->joins.size() < b->sims.size()) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return bfail(b, MITHRA_ECUDA, "event creation failed");
    b->joins.push_back(e);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(b, MITHRA_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  mithra_status st = MITHRA_OK;
  cudaEventRecord(b->fork, b->stream);
  for (size_t k = 0; k < b->sims.size() && st == MITHRA_OK; ++k) {
    mithra_sim* s = b->sims[k];
    cudaStreamWaitEvent(s->stream, b->fork, 0);
    const bool prof = s->profiling;
    s->profiling = false;
    for (int t = 0; t < 2 && st == MITHRA_OK; ++t) {
      st = with_types(s->prec, [&](auto tt, auto uu) {
        TYPES_OF(tt, uu);
        return launch_step<T, U>(s);
      });
    }
    s->profiling = prof;
    cudaEventRecord(b->joins[k], s->stream);
    cudaStreamWaitEvent(b->stream, b->joins[k], 0);
  }
  e = cudaStreamEndCapture(b->stream, &graph);
  if (st != MITHRA_OK) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, st, "capture of a member's step failed");
  }
  if (e != cudaSuccess) return bfail(b, MITHRA_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, MITHRA_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  b->dirty = false;
  return MITHRA_OK;
}

}  // namespace

extern "C" {

mithra_status mithra_batch_create(void* cuda_stream, mithra_batch** out) {
  if (!out) return bfail(nullptr, MITHRA_EINVAL, "out is NULL");
  *out = nullptr;
  mithra_batch* b = new (std::nothrow) mithra_batch();
  if (!b) return bfail(nullptr, MITHRA_ENOMEM, "host allocation failed");
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return bfail(nullptr, MITHRA_ECUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return bfail(nullptr, MITHRA_ECUDA, "event creation failed");
  }
  *out = b;
  return MITHRA_OK;
}

mithra_status mithra_batch_add(mithra_batch* b, mithra_sim* s) {
  if (!b || !s) return bfail(b, MITHRA_EINVAL, "batch or sim is NULL");
  if (s->in_batch) return bfail(b, MITHRA_EBUSY, "sim already belongs to a batch");
  if (s->stream == b->stream || s->stream == nullptr ||
      s->stream == reinterpret_cast<cudaStream_t>(1) || s->stream == reinterpret_cast<cudaStream_t>(2))
    return bfail(b, MITHRA_EINVAL, "a batched sim needs its own non-default stream");
  // work already queued on the sim's stream comes before the batch's work
  cudaEvent_t e;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
    return bfail(b, MITHRA_ECUDA, "event creation failed");
  cudaEventRecord(e, s->stream);
  cudaStreamWaitEvent(b->stream, e, 0);
  cudaEventDestroy(e);
  b->sims.push_back(s);
  s->in_batch = b;
  drop_step_graphs(s);
  drop_graph(b);
  return MITHRA_OK;
}

mithra_status mithra_batch_remove(mithra_batch* b, mithra_sim* s) {
  if (!b || !s) return bfail(b, MITHRA_EINVAL, "batch or sim is NULL");
  for (size_t k = 0; k < b->sims.size(); ++k) {
    if (b->sims[k] == s) {
      // later work on the sim's own stream waits for the batch
      cudaEvent_t e;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(e, b->stream);
        cudaStreamWaitEvent(s->stream, e, 0);
        cudaEventDestroy(e);
      }
      b->sims.erase(b->sims.begin() + (long)k);
      s->in_batch = nullptr;
      drop_graph(b);
      return MITHRA_OK;
    }
  }
  return bfail(b, MITHRA_EINVAL, "sim is not in this batch");
}

mithra_status mithra_batch_step(mithra_batch* b, int64_t n) {
  if (!b) return bfail(nullptr, MITHRA_EINVAL, "batch is NULL");
  if (n < 0) return bfail(b, MITHRA_EINVAL, "n must be >= 0");
  if (b->sims.empty() || n == 0) return MITHRA_OK;
  if (n >= 2 && (b->dirty || !b->exec)) {
    mithra_status st = capture(b);
    if (st != MITHRA_OK) return st;
  }
  while (b->joins.size() < b->sims.size()) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return bfail(b, MITHRA_ECUDA, "event creation failed");
    b->joins.push_back(e);
  }
  // work queued on a member's own stream comes before the batch's
  for (size_t k = 0; k < b->sims.size(); ++k) {
    cudaEventRecord(b->joins[k], b->sims[k]->stream);
    cudaStreamWaitEvent(b->stream, b->joins[k], 0);
  }
  for (int64_t t = 0; t + 1 < n; t += 2) {
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return bfail(b, MITHRA_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    for (mithra_sim* s : b->sims) s->n_issued += 2;
  }
  if (n % 2) {
    // one more step for every member, outside the graph
    cudaEventRecord(b->fork, b->stream);
    for (size_t k = 0; k < b->sims.size(); ++k) {
      mithra_sim* s = b->sims[k];
      cudaStreamWaitEvent(s->stream, b->fork, 0);
      mithra_status st = launch_one_step(s);
      if (st != MITHRA_OK) return bfail(b, st, s->err);
      if (b->joins.size() <= k) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
          return bfail(b, MITHRA_ECUDA, "event creation failed");
        b->joins.push_back(e);
      }
      cudaEventRecord(b->joins[k], s->stream);
      cudaStreamWaitEvent(b->stream, b->joins[k], 0);
    }
    drop_graph(b);  // members' parities changed
  }
  // later work on a member's own stream waits for the batch
  cudaEventRecord(b->done, b->stream);
  for (mithra_sim* s : b->sims) cudaStreamWaitEvent(s->stream, b->done, 0);
  return MITHRA_OK;
}

mithra_status mithra_batch_sync(mithra_batch* b) {
  if (!b) return bfail(nullptr, MITHRA_EINVAL, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, MITHRA_ECUDA, std::string("synchronize: ") + cudaGetErrorString(e));
  for (mithra_sim* s : b->sims) {
    mithra_status st = sync_status(s, true);
    if (st != MITHRA_OK) return bfail(b, st, s->err);
  }
  return MITHRA_OK;
}

mithra_status mithra_batch_set_mode(mithra_batch* b, int32_t fused) {
  if (!b) return bfail(nullptr, MITHRA_EINVAL, "batch is NULL");
  if (fused < 0 || fused > 2) return bfail(b, MITHRA_EINVAL, "mode must be 0, 1 or 2");
  if (b->mode != fused) {
    b->mode = fused;
    drop_graph(b);
  }
  return MITHRA_OK;
}

mithra_status mithra_batch_get_mode(const mithra_batch* b, int32_t* fused) {
  if (!b || !fused) return bfail(nullptr, MITHRA_EINVAL, "batch or out is NULL");
  *fused = b->fused_now ? 1 : 0;
  return MITHRA_OK;
}

mithra_status mithra_batch_stats(const mithra_batch* b, int64_t* captures,
                                 int64_t* fused_captures, double* capture_seconds) {
  if (!b) return bfail(nullptr, MITHRA_EINVAL, "batch is NULL");
  if (captures) *captures = b->captures;
  if (fused_captures) *fused_captures = b->fused_captures;
  if (capture_seconds) *capture_seconds = b->capture_s;
  return MITHRA_OK;
}

int32_t mithra_batch_size(const mithra_batch* b) { return b ? (int32_t)b->sims.size() : 0; }

const char* mithra_batch_last_error(const mithra_batch* b) {
  return b ? b->err.c_str() : g_thread_err.c_str();
}

mithra_status mithra_batch_destroy(mithra_batch* b) {
  if (!b) return MITHRA_OK;
  cudaStreamSynchronize(b->stream);
  for (mithra_sim* s : b->sims) s->in_batch = nullptr;
  drop_graph(b);
  if (b->d_table) cudaFree(b->d_table);
  if (b->d_blk) cudaFree(b->d_blk);
  if (b->d_pref) cudaFree(b->d_pref);
  if (b->d_zblk) cudaFree(b->d_zblk);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return MITHRA_OK;
}

}  // extern "C"
