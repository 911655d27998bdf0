// gpd_inst.cu -- explicit instantiation of the particle kernel (and, for the
// fixed-point deposit, the current reduction) for one mode count and deposit
// variant.  The build compiles this file once per pair, with GPD_NP (2M+1
// parts: 1, 3, 5, 7) and GPD_FA (1: float-atomic deposit) defined, so the
// instantiations compile in parallel.
#include "gpd.cuh"

#if !defined(GPD_NP) || !defined(GPD_FA)
#error "define GPD_NP and GPD_FA"
#endif

namespace qpic {

template <int NP, bool FA>
bool gpd_run(qpic_ctx *c, const PArgs &a, int grid, int ntiles, int chunk)
{
    return gpd_dispatch_tile<NP, FA>(c, a, grid, ntiles, chunk);
}
template bool gpd_run<GPD_NP, (GPD_FA != 0)>(qpic_ctx *, const PArgs &, int, int, int);

#if GPD_FA == 0
template <int NP>
void jreduce_run(qpic_ctx *c, const PArgs &a, int tiles_ok)
{
    jreduce_dispatch<NP>(c, a, tiles_ok);
}
template void jreduce_run<GPD_NP>(qpic_ctx *, const PArgs &, int);
#endif

}  // namespace qpic
