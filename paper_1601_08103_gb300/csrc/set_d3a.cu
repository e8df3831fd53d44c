// Kernels and launchers of the seven-velocity 3D sets (Secs. 8.3.1, 8.3.2) and D3Q9.
#include "set_impl.cuh"

namespace lee {
extern const SetOps kOpsD3Q7 = SetImpl<D3Q7>::make();
extern const SetOps kOpsD3Q7Di = SetImpl<D3Q7Di>::make();
extern const SetOps kOpsD3Q9 = SetImpl<D3Q9>::make();
}  // namespace lee
