// Host check of the double-float arithmetic in csrc/df64.cuh: prints inputs
// and results as exact float hex so that tests/test_df64.py can compare them
// with exact rational arithmetic.
#include <cstdio>
#include <cstdint>
#include <cmath>

#include "df64.cuh"

using namespace sdmd;

static uint64_t st = 0x9E3779B97F4A7C15ULL;
static double rnd() {   // xorshift64*, uniform-ish doubles in [-1, 1) times a random scale
  st ^= st >> 12; st ^= st << 25; st ^= st >> 27;
  const uint64_t r = st * 0x2545F4914F6CDD1DULL;
  const double u = (double)(r >> 11) / 9007199254740992.0 * 2.0 - 1.0;
  st ^= st >> 12; st ^= st << 25; st ^= st >> 27;
  const int e = (int)((st * 0x2545F4914F6CDD1DULL) >> 59) - 16;   // 2^-16 .. 2^15
  return std::ldexp(u, e);
}

static void pr(const char* op, dd a, dd b, dd r) {
  std::printf("%s %a %a %a %a %a %a\n", op, a.hi, a.lo, b.hi, b.lo, r.hi, r.lo);
}

int main() {
  for (int i = 0; i < 4000; ++i) {
    const double x = rnd(), y = rnd();
    const dd a = dd_from_double(x), b = dd_from_double(y);
    std::printf("from %a %a %a\n", x, a.hi, a.lo);
    pr("add", a, b, dd_add(a, b));
    pr("sub", a, b, dd_sub(a, b));
    pr("mul", a, b, dd_mul(a, b));
    if (b.hi != 0.f) pr("div", a, b, dd_div(a, b));
    if (b.hi != 0.f) pr("recip", b, b, dd_recip(b));
    const dd aa = dd_abs(a);
    pr("sqrt", aa, aa, dd_sqrt(aa));
    const dd c = dd_from_double(rnd());
    const dd f = dd_fma(a, b, c);
    std::printf("fma %a %a %a %a %a %a %a %a\n", a.hi, a.lo, b.hi, b.lo, c.hi, c.lo, f.hi, f.lo);
    // near-cancellation: a - (a + tiny)
    const dd t = dd_add(a, dd_from_double(x * 1e-9));
    pr("sub", a, t, dd_sub(a, t));
  }
  const long long ints[] = {0LL, 1LL, -7LL, 255LL * 255LL * 6220800LL, (1LL << 47) + 12345LL, -(1LL << 40) - 3LL};
  for (long long v : ints) {
    const dd d = dd_from_ll(v);
    std::printf("ll %lld %a %a\n", v, d.hi, d.lo);
  }
  return 0;
}
