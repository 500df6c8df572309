// Host check of rs::dmul_int (the integer-pipe FP64 product) against the
// host CPU's IEEE double multiply (round to nearest even), bit for bit.
// Built with nvcc as host code by tests/test_intmul_host.py.
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <random>
#include "rs_wave.cuh"
int main() {
  std::mt19937_64 g(1);
  long long bad = 0, tested = 0, special = 0;
  auto check = [&](double a, double b) {
    bool sp; double r = rs::dmul_int(a, b, sp);
    if (sp) { ++special; return; }
    volatile double va = a, vb = b; double ref = va * vb;
    ++tested;
    if (rs::bits_of(r) != rs::bits_of(ref)) { if (bad < 10) printf("MISMATCH a=%a b=%a got=%a ref=%a\n", a, b, r, ref); ++bad; }
  };
  for (long long i = 0; i < 20000000; ++i) {
    unsigned long long ua = g(), ub = g();
    double a = rs::double_of(ua), b = rs::double_of(ub);
    check(a, b);
    // rotation-like magnitudes
    std::uniform_real_distribution<double> u(-1, 1); std::normal_distribution<double> nrm;
    check(u(g), nrm(g));
    // mantissa edge cases: all ones / few bits
    unsigned long long m1 = g() & 0xfffffffffffffull, m2 = g() & 0xfffffffffffffull;
    int sh = g() % 53; m1 |= (1ull << sh) - 1; m2 &= ~((1ull << (g() % 53)) - 1);
    check(rs::double_of((1023ull << 52) | m1), rs::double_of((1023ull << 52) | m2));
  }
  // exact halfway cases: (1 + 2^-26)^2 style and powers of two, near over/underflow
  for (int e = -1100; e <= 1100; e += 7) for (int k = 0; k < 60; ++k) {
    double a = std::ldexp(1.0 + std::ldexp(1.0, -k % 53), e / 2), b = std::ldexp(1.0 + std::ldexp(3.0, -(k % 50)), e - e / 2);
    check(a, b); check(-a, b); check(a, std::nextafter(b, 2 * b));
  }
  printf("tested=%lld special=%lld bad=%lld\n", tested, special, bad);
  return bad != 0;
}
