// Host check of the fixed-point tally arithmetic (tally_fixed.cuh): reads
// lines "v" (signed 64-bit values) from stdin, adds them to a 128-bit
// accumulator with fixed128_hi_inc, and prints the final words and
// fixed128_value of the sum.
#include <cstdio>

#include "../../paper_2307_11107_gb300/csrc/tally_fixed.cuh"

int main() {
  unsigned long long lo = 0, hi = 0;
  long long v;
  while (std::scanf("%lld", &v) == 1) {
    hi += apic::fixed128_hi_inc(lo, v);
    lo += (unsigned long long)v;
  }
  std::printf("%llu %llu %.17g\n", lo, hi, apic::fixed128_value(lo, hi));
  return 0;
}
