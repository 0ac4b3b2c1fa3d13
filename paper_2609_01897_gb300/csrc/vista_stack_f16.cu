// Instantiations of the mixed-precision stacking kernel for FP16-pair visibilities.
#include "vista_stack.cuh"

namespace vista {

cudaError_t launch_mixed_f16(const RunArgs &a, int ns, int pf, int npol, int wpc, cudaStream_t st)
{
    return launch_mixed_vt<VISTA_VIS_F16X2>(a, ns, pf, npol, wpc, st);
}

}  // namespace vista
