// Launch profile hooks (see kr_profile.cu).
#pragma once

#include <cuda_runtime.h>

#include "kr_rows.cuh"

namespace kr {

enum KernelClass : int {
  KC_SPMM = 0, KC_LINCOMB = 1, KC_REDUCE = 2, KC_COEF = 3, KC_OTHER = 4, KC_SPMM32 = 5, KC_LINCOMB32 = 6
};

struct ProfToken {
  int cls = 0;
  cudaEvent_t a = nullptr;
  bool active = false;
};

ProfToken prof_begin(int cls, cudaStream_t st);
bool prof_active();  // launch counting (and timing) on
void prof_end(ProfToken& t, cudaStream_t st, double flops, double bytes);

double red_flops(const RedSet& rs, int64_t n, int s);
double red_bytes(const RedSet& rs, int64_t n, int s, double elem, const void* const* counted, int ncounted);

}  // namespace kr
