// Modal prolongation launcher (prolong.cu).
#pragma once

#include "internal.h"

namespace cheb {

int check_prolong_pair(const cheb_plan_s* coarse, const cheb_plan_s* fine);
// uf = prolongation of uc; s1, s2: scratch arrays of at least
// nx_f ny_f nz_c elements (the intermediate after the x and y passes)
template <typename T>
int launch_prolong(const cheb_plan_s* coarse, const cheb_plan_s* fine, const T* uc, T* uf, T* s1,
                   T* s2, cudaStream_t s);

}  // namespace cheb
