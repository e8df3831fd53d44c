// Kernels and launchers of the 1D and 2D velocity sets (Secs. 8.1, 8.2).
#include "set_impl.cuh"

namespace lee {
extern const SetOps kOpsD1Q3 = SetImpl<D1Q3>::make();
extern const SetOps kOpsD2Q5 = SetImpl<D2Q5>::make();
extern const SetOps kOpsD2Q5Di = SetImpl<D2Q5Di>::make();
}  // namespace lee
