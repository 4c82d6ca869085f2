// kt_oracle_flops.cpp -- the oracle (kt_oracle.c) compiled with the operation-counting scalar of
// flops.hpp in place of double: the algorithmic operation count of the scheme per cell, from the
// same code the parity tests trust.  TEST AND MEASUREMENT INFRASTRUCTURE ONLY.
//
// Built single-threaded (no OpenMP), like the plain oracle with -ffp-contract=off, so its
// results equal the plain oracle's bit for bit.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "flops.hpp"

unsigned long long ko_flop_count[FK_N] = {};

#define double fdouble
#include "kt_oracle.c"
#undef double

extern "C" {
// Copy the counters (add/sub, mul, div, sqrt, exp/log/pow/tanh, compares) into out[6]; zero
// them if reset is non-zero.
void ko_flops_read(unsigned long long* out, int reset) {
  for (int k = 0; k < FK_N; ++k) {
    out[k] = ko_flop_count[k];
    if (reset) ko_flop_count[k] = 0;
  }
}
}
