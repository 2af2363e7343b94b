// bunch.cu -- host-side generator of a macroparticle bunch in the rest frame
// (Sec. "Electron Bunch Generation"): uniform numbers from the Halton
// sequence (or a counter-based pseudo-random generator) mapped to a uniform
// longitudinal profile (Eq. uniform1D), Gaussian transverse positions and
// momenta by the Box-Muller transformation (Eq. gaussian1D, Eq. gaussian2D),
// truncation at a distance from the bunch centre (input group
// bunch-initialization, transverse-truncation), the split-Gaussian head and
// tail that smooth a uniform current profile, and the longitudinal
// displacement that sets an initial bunching factor (Eq. bunchingFactor, in
// the reading dz = -(2 bf / kb) sin(kb z) of the garbled print).  No GPU is
// involved.
#include <cmath>
#include <cstdint>
#include <string>

#include "mithra.h"

namespace mithra {
void set_thread_error(const std::string& msg);  // mithra_last_error(NULL)
}

namespace {

constexpr double kPiB = 3.14159265358979323846;

// Radical inverse of index i in base b: the digits of i in base b mirrored
// about the radix point (one dimension of the Halton sequence).
double radical_inverse(uint64_t i, uint32_t b) {
  double x = 0.0, f = 1.0 / b;
  while (i > 0) {
    x += f * (double)(i % b);
    i /= b;
    f /= b;
  }
  return x;
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", 2014): a 64-bit mix of a counter, used here counter-based.
uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Nine uniform numbers in (0, 1) per draw: the Halton point of index
// draw + 1 in the first nine prime bases (index 0 would give 0 in every
// base), or the counter-based generator at (seed, draw, dimension).
// Dimensions: 0, 1 transverse position (Box-Muller radius, angle); 2 the
// uniform z; 3, 4 the Gaussian of the head and tail; 5, 6 the transverse
// momenta; 7, 8 the longitudinal momentum.
constexpr int kDims = 9;
const uint32_t kPrimes[kDims] = {2, 3, 5, 7, 11, 13, 17, 19, 23};

void uniforms(int sequence, uint64_t seed, uint64_t draw, double u[kDims]) {
  for (int d = 0; d < kDims; ++d) {
    if (sequence == 1) {
      u[d] = radical_inverse(draw + 1, kPrimes[d]);
    } else {
      const uint64_t r = splitmix64(splitmix64(seed ^ (0xD1B54A32D192ED03ull * (d + 1))) + draw);
      u[d] = ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0);  // 2^-53 grid, never 0
    }
  }
}

mithra_status bad(const char* msg) {
  mithra::set_thread_error(msg);
  return MITHRA_EINVAL;
}

}  // namespace

extern "C" mithra_status mithra_make_bunch(const mithra_bunch_spec* s, double* x, double* y,
                                          double* z, double* ux, double* uy, double* uz,
                                          double* q_macro) {
  if (!s || !x || !y || !z || !ux || !uy || !uz) return bad("spec and arrays must not be NULL");
  if (s->n < 1) return bad("n must be >= 1");
  if (!(s->z_hi >= s->z_lo)) return bad("z_hi must be >= z_lo");
  if (s->sigma_x < 0 || s->sigma_y < 0 || s->ux_sigma < 0 || s->uy_sigma < 0 ||
      s->uz_sigma < 0 || s->taper_sigma < 0)
    return bad("spreads must be >= 0");
  if (s->sequence != 0 && s->sequence != 1) return bad("sequence must be 0 or 1");
  if (s->bf < 0 || s->bf >= 1) return bad("bunching factor must be in [0, 1)");
  if (s->bf > 0 && !(s->kb > 0)) return bad("a bunching factor needs kb > 0");
  const double L = s->z_hi - s->z_lo;
  const double tail = s->taper_sigma > 0 ? std::sqrt(2.0 * kPiB) * s->taper_sigma : 0.0;
  // particles of the uniform part; the others form the split Gaussian of the
  // same peak density at the head and tail
  const int64_t n = s->n;
  const int64_t n_uni = (L + tail) > 0 ? (int64_t)std::llround((double)n * L / (L + tail)) : n;
  const double R = s->trunc_r;
  uint64_t draw = 0;
  const uint64_t max_draws = (uint64_t)n * 1000 + 1000;
  for (int64_t p = 0; p < n; ++p) {
    double u[kDims];
    double xr, yr;
    for (;;) {  // transverse truncation by rejection, Eq. gaussian2D
      if (draw >= max_draws) return bad("truncation rejects nearly every draw");
      uniforms(s->sequence, s->seed, draw++, u);
      const double r = std::sqrt(-2.0 * std::log(u[0]));
      xr = r * std::cos(2.0 * kPiB * u[1]);
      yr = r * std::sin(2.0 * kPiB * u[1]);
      const double dx = s->sigma_x * xr, dy = s->sigma_y * yr;
      if (R <= 0 || dx * dx + dy * dy <= R * R) break;
    }
    x[p] = s->x0 + s->sigma_x * xr;
    y[p] = s->y0 + s->sigma_y * yr;
    double zz;
    if (p < n_uni) {
      zz = s->z_lo + L * u[2];  // Eq. uniform1D with total width L
    } else {
      // the split Gaussian: its lower half behind the tail, the upper half
      // ahead of the head (Eq. gaussian1D)
      const double g = s->taper_sigma * std::sqrt(-2.0 * std::log(u[3])) *
                       std::cos(2.0 * kPiB * u[4]);
      zz = g < 0 ? s->z_lo + g : s->z_hi + g;
    }
    if (s->bf > 0) zz -= (2.0 * s->bf / s->kb) * std::sin(s->kb * zz);
    z[p] = zz;
    // momenta: Eq. gaussian2D for the transverse pair, Eq. gaussian1D for u_z
    const double rm = std::sqrt(-2.0 * std::log(u[5]));
    ux[p] = s->ux_sigma * rm * std::cos(2.0 * kPiB * u[6]);
    uy[p] = s->uy_sigma * rm * std::sin(2.0 * kPiB * u[6]);
    uz[p] = s->uz_mean + s->uz_sigma * std::sqrt(-2.0 * std::log(u[7])) *
                             std::cos(2.0 * kPiB * u[8]);
  }
  if (q_macro) *q_macro = -s->charge / (double)n;
  return MITHRA_OK;
}
