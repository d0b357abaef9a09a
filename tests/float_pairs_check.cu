// Host check of the library's integer-arithmetic conversions between
// doubles, floats and (hi, lo) float pairs (csrc/dfloat.cuh) against the
// IEEE conversions they stand in for.  Built with nvcc as host code and
// run by test_float_pairs.py; prints the mismatch counts, exits 1 on any.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../paper_2101_08453_gb300/csrc/dfloat.cuh"

using namespace mcw;

static bool same(double a, double b) { return std::memcmp(&a, &b, 8) == 0; }
static bool same(float a, float b) { return std::memcmp(&a, &b, 4) == 0; }

int main(int argc, char** argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 2000000;
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  long bad_p2d = 0, bad_f = 0, bad_split = 0;
  for (long t = 0; t < n; ++t) {
    // pair_to_double == (double)hi + (double)lo on normalized pairs, with
    // powers of two for hi (the borrow case) and exact half-unit ties
    const int ex = (int)(rng() % 160) - 60;
    float hi, lo;
    switch (t % 4) {
      case 0: {
        const double x = std::ldexp(U(rng), ex);
        hi = (float)x;
        lo = (float)(x - (double)hi);
        break;
      }
      case 1:
        hi = std::ldexp(U(rng) < 0.0 ? -1.0f : 1.0f, ex);
        lo = (float)(U(rng) * std::ldexp(0.5, std::ilogb(hi) - 23));
        break;
      case 2: {
        hi = (float)std::ldexp(U(rng), ex);
        const long long k = (long long)(U(rng) * (1 << 27));
        lo = (float)((k + 0.5) * std::ldexp(1.0, std::ilogb(hi) - 52));
        break;
      }
      default:
        hi = (float)std::ldexp(U(rng), ex);
        lo = (float)std::ldexp(U(rng), std::ilogb(hi) - 24 - (int)(rng() % 40));
        break;
    }
    if (t % 50 == 0) {  // the four signed-zero pairs
      hi = (t % 100) ? 0.0f : -0.0f;
      lo = (t % 200 < 100) ? 0.0f : -0.0f;
    }
    if (!same(pair_to_double(hi, lo), (double)hi + (double)lo)) ++bad_p2d;
    // float_of_bits == (float)x: random bit patterns, scaled values, ties
    double x;
    if (t % 3 == 0) {
      const unsigned long long u = rng();
      std::memcpy(&x, &u, 8);
    } else if (t % 3 == 1) {
      x = std::ldexp(U(rng), (int)(rng() % 300) - 150);
    } else {
      const float f = (float)std::ldexp(U(rng), (int)(rng() % 250) - 125);
      x = (double)f + std::ldexp(1.0, std::ilogb(f) - 24) * ((rng() & 1) ? 1.0 : -1.0);
    }
    const float want = (float)x, got = float_of_bits(x);
    if (!(std::isnan(want) && std::isnan(got)) && !same(want, got)) ++bad_f;
    // split_bits: hi + lo within 2^-48 |x|, |lo| <= ulp(hi)/2, zero exact
    const double y = (t % 11 == 0) ? ((t % 22) ? 0.0 : -0.0) : std::ldexp(U(rng), (int)(rng() % 165) - 69);
    const float2 p = split_bits(y);
    const bool ok = y == 0.0 ? (p.y == 0.0f && p.x == 0.0f && std::signbit(p.x) == std::signbit(y))
                             : (std::fabs((double)p.x + (double)p.y - y) <= std::ldexp(std::fabs(y), -48) &&
                                std::fabs(p.y) <= std::ldexp(std::fabs(p.x), -24));
    if (!ok) ++bad_split;
  }
  // float_of_i29 == (float)r over the whole range |r| < 2^29 in strides,
  // and every value near the rounding boundaries of the top binades
  long bad_i = 0;
  for (long r = -(1L << 29) + 1; r < (1L << 29); r += 997)
    if (!same(float_of_i29((int)r), (float)r)) ++bad_i;
  for (int e = 24; e <= 28; ++e)
    for (long c = -64; c <= 64; ++c)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        const long r = sgn * ((1L << e) + c * 3);
        if (r > -(1L << 29) && r < (1L << 29) && !same(float_of_i29((int)r), (float)r)) ++bad_i;
      }
  std::printf("pair_to_double %ld float_of_bits %ld split_bits %ld of %ld, float_of_i29 %ld\n",
              bad_p2d, bad_f, bad_split, n, bad_i);
  return (bad_p2d || bad_f || bad_split || bad_i) ? 1 : 0;
}
