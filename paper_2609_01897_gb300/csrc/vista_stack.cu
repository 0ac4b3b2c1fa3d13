// Dispatch of the mixed-precision stacking kernel by launch class (the
// kernel is in vista_stack.cuh, its instantiations in vista_stack_<type>.cu).
#include "vista_stack.cuh"

namespace vista {

cudaError_t launch_mixed(const RunArgs &a, int key, int wpc, int prefetch, cudaStream_t st)
{
    const int npol = key & 0xff, ns = (key >> 8) & 0xff, vt = key >> 16;
    switch (vt) {
    case VISTA_VIS_C64: return launch_mixed_c64(a, ns, prefetch, npol, wpc, st);
    case VISTA_VIS_C128: return launch_mixed_c128(a, ns, prefetch, npol, wpc, st);
    case VISTA_VIS_F16X2: return launch_mixed_f16(a, ns, prefetch, npol, wpc, st);
    case VISTA_VIS_BF16X2: return launch_mixed_bf16(a, ns, prefetch, npol, wpc, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vista
