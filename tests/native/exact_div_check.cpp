// Host driver for the integer quotient rounding of the score kernel: reads "c L" pairs from
// standard input and prints the bits of RN(c / L) as 16 hex digits, one line per pair.
#include <cinttypes>
#include <cstdio>

#include "exact_div.h"

int main() {
  unsigned long long c, L;
  while (std::scanf("%llu %llu", &c, &L) == 2) {
    const ace::DivConst k = ace::make_div_const(static_cast<uint32_t>(L));
    std::printf("%016" PRIx64 "\n", ace::rn_quotient_bits(static_cast<uint32_t>(c), k));
  }
  return 0;
}
