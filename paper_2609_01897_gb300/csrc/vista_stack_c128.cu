// Instantiations of the mixed-precision stacking kernel for complex128 visibilities.
#include "vista_stack.cuh"

namespace vista {

cudaError_t launch_mixed_c128(const RunArgs &a, int ns, int pf, int npol, int wpc, cudaStream_t st)
{
    return launch_mixed_vt<VISTA_VIS_C128>(a, ns, pf, npol, wpc, st);
}

}  // namespace vista
