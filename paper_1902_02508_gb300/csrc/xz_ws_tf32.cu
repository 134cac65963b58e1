// TF32X2 instantiations of the warp-specialised tensor-core x-z kernel
// (xz_ws.cuh); the host side and the BF16X3 instantiations are in xz_ws.cu.
#include "eles_internal.h"
#include "xz_ws.cuh"

namespace eles {

cudaError_t ws_launch_tf32(const ws::WsMulti &m, int nz, int opc, cudaStream_t st)
{
    using namespace ws;
#define ELES_WS_GO(NZ)                                                                                   \
    if (nz == NZ) return opc == 2 ? ws_launch<NZ, MODE_TF32X2, 2>(m, st) : ws_launch<NZ, MODE_TF32X2, 1>(m, st);
    ELES_WS_NZ_LIST(ELES_WS_GO)
#undef ELES_WS_GO
    return cudaErrorInvalidValue;
}

}  // namespace eles
