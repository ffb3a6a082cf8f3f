// Modal prolongation launcher (prolong.cu).
#pragma once

#include "internal.h"

namespace cheb {

int check_prolong_pair(const cheb_plan_s* coarse, const cheb_plan_s* fine);
// uf = prolongation of uc; s1, s2: scratch arrays of at least fine->size()/2 + 1 elements
template <typename T>
int launch_prolong(const cheb_plan_s* coarse, const cheb_plan_s* fine, const T* uc, T* uf, T* s1,
                   T* s2, cudaStream_t s);

}  // namespace cheb
