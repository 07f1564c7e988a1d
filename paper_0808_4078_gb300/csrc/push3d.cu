// push3d.cu -- fused 3D3V particle step (gather, Boris, drag, move, Esirkepov deposit).
#include "pic_internal.cuh"

namespace pic {

bool has_push3d() { return false; }

cudaError_t launch_push3d(const Args&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace pic
