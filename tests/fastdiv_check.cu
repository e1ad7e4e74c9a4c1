// Host-only check of the invariant-divisor division used for node indices
// (FastDiv in albm_node.cuh): fdiv(n, make_fastdiv(d)) == n / d for the
// divisors and numerators listed below, including 1, powers of two and
// their neighbours, and the largest 32-bit values.  Prints the number of
// mismatches; exit status 0 when there are none.
#include <cstdio>
#include <cstdint>
#include <vector>

#include "../paper_1501_04741_gb300/csrc/albm_node.cuh"

int main() {
  std::vector<unsigned> ds;
  for (unsigned d = 1; d <= 4096; ++d) ds.push_back(d);
  for (int k = 12; k < 32; ++k) {
    const unsigned p = 1u << k;
    ds.push_back(p - 1);
    ds.push_back(p);
    ds.push_back(p + 1);
    ds.push_back(p + 12345u);
  }
  ds.push_back(0xffffffffu);
  ds.push_back(0xfffffffeu);
  ds.push_back(1000003u);
  std::vector<unsigned> ns;
  for (unsigned n = 0; n < 20000; ++n) ns.push_back(n);
  uint64_t x = 88172645463325252ull;   // xorshift64 (Marsaglia 2003)
  for (int i = 0; i < 20000; ++i) {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    ns.push_back((unsigned)x);
  }
  for (unsigned n = 0xffffffffu - 5000u; n != 0; ++n) ns.push_back(n);
  long long bad = 0, checked = 0;
  for (unsigned d : ds) {
    const albm::FastDiv f = albm::make_fastdiv(d);
    for (unsigned n : ns) {
      // multiples of d and their neighbours, where a wrong rounding shows
      const unsigned q = n / d;
      const unsigned cand[3] = {n, q * d, q * d + (d - 1)};
      for (unsigned c : cand) {
        ++checked;
        if (albm::fdiv(c, f) != c / d) {
          if (bad < 10) printf("mismatch d=%u n=%u got %u want %u\n", d, c, albm::fdiv(c, f), c / d);
          ++bad;
        }
      }
    }
  }
  printf("checked %lld mismatches %lld\n", checked, bad);
  return bad == 0 ? 0 : 1;
}
