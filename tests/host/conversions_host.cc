// The integer conversions of hweno_state.cuh (widen_f, narrow_exact, narrow_trunc)
// against the host's own conversions, for every float bit pattern: widen_f(x) equals
// (double)x bit for bit (NaN: a NaN with x's sign and payload), narrow_exact returns x
// from it; and narrow_trunc on doubles around every float binade, from subnormal to
// beyond the float range, against a truncation toward zero written with the host's
// rounding mode.  Prints the number of mismatches of each check.
#include <cfenv>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "shim.h"
#include "hweno_state.cuh"

using namespace hw;

static uint64_t dbits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
static uint32_t fbits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }
static float fof(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static double dof(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }

int main() {
  long long bad_widen = 0, bad_round = 0, bad_trunc = 0, n_trunc = 0;
  for (uint64_t u = 0; u <= 0xffffffffull; u++) {
    const float x = fof((uint32_t)u);
    const double w = widen_f(x);
    if (std::isnan(x)) {
      const uint64_t wb = dbits(w);
      if (!std::isnan(w) || (wb >> 63) != (u >> 31) || ((wb >> 29) & 0x7fffff) != (u & 0x7fffff)) bad_widen++;
    } else if (dbits(w) != dbits((double)x)) {
      bad_widen++;
    }
    if (fbits(narrow_exact(w)) != (uint32_t)u) bad_round++;
  }
  // truncation toward zero of doubles: the host's conversion under FE_TOWARDZERO
  fesetround(FE_TOWARDZERO);
  uint64_t state = 88172645463325252ull;
  for (int E = 0; E < 2047; E++)
    for (int k = 0; k < 4096; k++) {
      state ^= state << 13; state ^= state >> 7; state ^= state << 17;
      const uint64_t b = ((uint64_t)(k & 1) << 63) | ((uint64_t)E << 52) | (state & 0xfffffffffffffull);
      const double y = dof(b);
      volatile double vy = y;
      const float ref = (float)vy;  // toward zero: overflow gives the largest float
      float got = narrow_trunc(y);
      n_trunc++;
      if (std::isinf(got) && !std::isinf(ref) && std::fabs(ref) == 3.4028234663852886e38f && std::fabs(y) > 3.4028234663852886e38)
        continue;  // beyond the float range narrow_trunc gives infinity
      if (fbits(got) != fbits(ref)) bad_trunc++;
    }
  fesetround(FE_TONEAREST);
  printf("widen %lld\nround_trip %lld\ntrunc %lld of %lld\n", bad_widen, bad_round, bad_trunc, n_trunc);
  return 0;
}
