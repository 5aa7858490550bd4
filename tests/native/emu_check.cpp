// Host check of the integer-pipe double products (fv_emu.h, without and with
// signed zeros on the fast path) against the host's IEEE-754 multiplication
// (round to nearest, ties to even).
// Prints "cases fast mismatches" and exits non-zero on any mismatch on the
// fast path.  Built and run by tests/test_emu_cpu.py.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "../../paper_2306_14011_gb300/csrc/fv_emu.h"

static uint64_t bits_of(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
static double of_bits(uint64_t b) { double x; std::memcpy(&x, &b, 8); return x; }

int main(int argc, char **argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 4000000;
  std::mt19937_64 rng(12345);
  long fast = 0, bad = 0, cases = 0;
  auto check = [&](uint64_t A, uint64_t B) {
    const double a = of_bits(A), b = of_bits(B);
    volatile double p = a * b;  // the host's IEEE product
    const uint64_t P = bits_of(p);
    ++cases;
    for (int variant = 0; variant < 2; ++variant) {
      uint32_t hr, lr;
      const uint32_t ha = (uint32_t)(A >> 32), la = (uint32_t)A, hb = (uint32_t)(B >> 32), lb = (uint32_t)B;
      const bool ok = variant == 0 ? fvk::emu_dmul_bits(ha, la, hb, lb, hr, lr)
                                   : fvk::emu_dmul_bits_z(ha, la, hb, lb, hr, lr);
      if (!ok) continue;
      if (variant == 0) ++fast;
      const uint64_t R = ((uint64_t)hr << 32) | lr;
      if (R != P) {  // the fast path never sees a NaN
        if (bad < 10) std::printf("variant %d mismatch %016llx * %016llx: %016llx vs %016llx\n", variant,
                                  (unsigned long long)A, (unsigned long long)B, (unsigned long long)R,
                                  (unsigned long long)P);
        ++bad;
      }
    }
  };
  for (long i = 0; i < n; ++i) {
    const int kind = (int)(i % 6);
    uint64_t A = rng(), B = rng();
    if (kind == 1) {  // exponents near the middle: ordinary products
      A = (A & 0x800fffffffffffffull) | ((uint64_t)(1023 + (int)(rng() % 64) - 32) << 52);
      B = (B & 0x800fffffffffffffull) | ((uint64_t)(1023 + (int)(rng() % 64) - 32) << 52);
    } else if (kind == 2) {  // short significands: exact products and ties to even
      A = (A & 0x8000000000000000ull) | ((uint64_t)(1023 + (int)(rng() % 16) - 8) << 52) |
          ((rng() & 0x7ffffffull) << 25);
      B = (B & 0x8000000000000000ull) | ((uint64_t)(1023 + (int)(rng() % 16) - 8) << 52) |
          ((rng() & 0x7ffffffull) << 25);
    } else if (kind == 3) {  // results near overflow and underflow
      const int ea = 1 + (int)(rng() % 2046);
      const int target = (rng() & 1) ? 2046 - (int)(rng() % 3) : 1 + (int)(rng() % 3);
      int eb = target - ea + 1023;
      eb = eb < 1 ? 1 : (eb > 2046 ? 2046 : eb);
      A = (A & 0x800fffffffffffffull) | ((uint64_t)ea << 52);
      B = (B & 0x800fffffffffffffull) | ((uint64_t)eb << 52);
    } else if (kind == 4) {  // zeros, subnormals, infinities and NaN mixed with ordinary values
      const uint64_t special[] = {0ull, 0x8000000000000000ull, 1ull, 0x000fffffffffffffull, 0x7ff0000000000000ull,
                                  0xfff0000000000000ull, 0x7ff8000000000000ull, 0x0010000000000000ull,
                                  0x7fefffffffffffffull, 0x3ff0000000000000ull};
      if (rng() & 1) A = special[rng() % 10];
      if (rng() & 1) B = special[rng() % 10];
    } else if (kind == 5) {  // all-ones and minimal significands (carry out of rounding)
      A = (A & 0x8000000000000000ull) | ((uint64_t)(1000 + (int)(rng() % 40)) << 52) |
          (0x000fffffffffffffull - (rng() & 0xff));
      B = (B & 0x8000000000000000ull) | ((uint64_t)(1000 + (int)(rng() % 40)) << 52) | (rng() & 0xff);
    }
    check(A, B);
  }
  std::printf("%ld %ld %ld\n", cases, fast, bad);
  return bad ? 1 : 0;
}
