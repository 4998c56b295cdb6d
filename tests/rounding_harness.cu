// Host harness for the exact-sum rounding of the tensor-core products: reads
// "hi lo e2" triples (decimal) from stdin and prints, per line, the bit
// pattern of round_hl(hi, lo, e2) -- (hi 2^24 + lo) 2^e2 rounded once to the
// nearest double, ties to even -- as 16 hex digits.  Built and driven by
// test_rounding.py, which checks every result against exact rational
// arithmetic.
#include <cstdio>
#include <cstring>

#include "../paper_2210_03714_gb300/csrc/ozaki.cuh"

int main() {
  long long hi, lo;
  int e2;
  while (std::scanf("%lld %lld %d", &hi, &lo, &e2) == 3) {
    const double v = fmk::oz::round_hl(hi, lo, e2);
    unsigned long long b;
    std::memcpy(&b, &v, sizeof b);
    std::printf("%016llx\n", b);
  }
  return 0;
}
