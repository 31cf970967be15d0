// ffs_decoder_stage.cu -- the one-stage-per-round decoder functions
// (stage_round), compiled once for every heap size the dispatchers use.
#define FFS_DECODER_BODIES
#include "ffs_device.cuh"

namespace fgpu {

#define FFS_STAGE_INST(MM)                                                                                          \
    template __device__ uint4 stage_round<MM, false, false>(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t,       \
                                                             const int16_t *, uint32_t, uint32_t, uint32_t);        \
    template __device__ uint4 stage_round<MM, false, true>(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t,        \
                                                            const int16_t *, uint32_t, uint32_t, uint32_t);         \
    template __device__ uint4 stage_round<MM, true, false>(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t,        \
                                                            const int16_t *, uint32_t, uint32_t, uint32_t);         \
    template __device__ uint4 stage_round<MM, true, true>(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t,         \
                                                           const int16_t *, uint32_t, uint32_t, uint32_t);
FFS_STAGE_INST(1) FFS_STAGE_INST(2) FFS_STAGE_INST(3) FFS_STAGE_INST(4) FFS_STAGE_INST(5) FFS_STAGE_INST(6)
FFS_STAGE_INST(7) FFS_STAGE_INST(8) FFS_STAGE_INST(9) FFS_STAGE_INST(10) FFS_STAGE_INST(11) FFS_STAGE_INST(12)
FFS_STAGE_INST(13) FFS_STAGE_INST(14) FFS_STAGE_INST(15) FFS_STAGE_INST(16) FFS_STAGE_INST(kMaxM)
#undef FFS_STAGE_INST

}  // namespace fgpu
