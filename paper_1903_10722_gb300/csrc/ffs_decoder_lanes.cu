// ffs_decoder_lanes.cu -- the stage-parallel decoder (lane_decode), compiled
// once for every heap size its dispatcher uses.
#define FFS_LANES_BODIES
#include "ffs_lanes.cuh"

namespace fgpu {

#define FFS_LANE_INST(MM)                                                                                           \
    template __device__ int32_t lane_decode<MM>(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, \
                                                uint32_t, uint32_t);
FFS_LANE_INST(1) FFS_LANE_INST(2) FFS_LANE_INST(3) FFS_LANE_INST(4) FFS_LANE_INST(5) FFS_LANE_INST(6)
FFS_LANE_INST(7) FFS_LANE_INST(8) FFS_LANE_INST(9) FFS_LANE_INST(10) FFS_LANE_INST(11) FFS_LANE_INST(12)
FFS_LANE_INST(13) FFS_LANE_INST(14) FFS_LANE_INST(15) FFS_LANE_INST(16) FFS_LANE_INST(kMaxM)
#undef FFS_LANE_INST

}  // namespace fgpu
