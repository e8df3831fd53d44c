// Kernels and launchers of the 3D edge sets D3Q13 and D3Q19 (Sec. 8.3.1).
#include "set_impl.cuh"

namespace lee {
extern const SetOps kOpsD3Q13 = SetImpl<D3Q13>::make();
extern const SetOps kOpsD3Q19 = SetImpl<D3Q19>::make();
}  // namespace lee
