// gpd_inst.cu -- explicit instantiation of the particle kernel (and, for the
// fixed-point deposit, the current reduction), or of the batched particle
// phase, for one mode count, deposit variant and set of tile shapes.  The
// build compiles this file once per group, with GPD_NP (2M+1 parts: 1, 3, 5,
// 7), GPD_FA (1: float-atomic deposit), GPD_BATCH (1: the batched phase) and
// GPD_SHAPES (bit k: tile shape k of 16x8, 32x8, 8x8, 16x16, 32x4) defined,
// so the instantiations compile in parallel.
#include "gpd.cuh"

#if !defined(GPD_NP) || !defined(GPD_FA) || !defined(GPD_BATCH) || !defined(GPD_SHAPES)
#error "define GPD_NP, GPD_FA, GPD_BATCH and GPD_SHAPES"
#endif

namespace qpic {

template <int NP, int TZ, int TR, bool FA>
void gpd_shape(qpic_ctx *c, const PArgs &a, int grid, int ntiles, int chunk)
{
    gpd_launch2<NP, TZ, TR, FA>(c, a, grid, ntiles, chunk);
}

template <int NP, int TZ, int TR>
void jreduce_shape(qpic_ctx *c, const PArgs &a, int tiles_ok)
{
    jreduce_launch<NP, TZ, TR>(c, a, tiles_ok);
}

template <int NP, int TZ, int TR>
void batch_shape(const BatchRun *runs, const int *tprefix, int nruns, int *head, const BatchCtl *ctl,
                 int blocks, cudaStream_t st)
{
    batch_particles_launch2<NP, TZ, TR>(runs, tprefix, nruns, head, ctl, blocks, st);
}

#if GPD_BATCH == 0
#if GPD_FA == 0
#define QPIC_INST_RED(TZ, TR) template void jreduce_shape<GPD_NP, TZ, TR>(qpic_ctx *, const PArgs &, int);
#else
#define QPIC_INST_RED(TZ, TR)
#endif
#define QPIC_INST(TZ, TR)                                                                            \
    template void gpd_shape<GPD_NP, TZ, TR, (GPD_FA != 0)>(qpic_ctx *, const PArgs &, int, int, int); \
    QPIC_INST_RED(TZ, TR)
#else
#define QPIC_INST(TZ, TR)                                                                \
    template void batch_shape<GPD_NP, TZ, TR>(const BatchRun *, const int *, int, int *, \
                                              const BatchCtl *, int, cudaStream_t);
#endif

#if GPD_SHAPES & 1
QPIC_INST(16, 8)
#endif
#if GPD_SHAPES & 2
QPIC_INST(32, 8)
#endif
#if GPD_SHAPES & 4
QPIC_INST(8, 8)
#endif
#if GPD_SHAPES & 8
QPIC_INST(16, 16)
#endif
#if GPD_SHAPES & 16
QPIC_INST(32, 4)
#endif

}  // namespace qpic
