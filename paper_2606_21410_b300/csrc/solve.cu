// Krylov workspace and solver drivers.
#include "internal.h"

namespace cheb {

struct Workspace {
  int dummy = 0;
};

void free_workspace(cheb_plan_s* p) {
  delete p->ws;
  p->ws = nullptr;
}

}  // namespace cheb
