// ffs_decoder_pair.cu -- the stage-pair decoder functions (pair_round),
// compiled once for every heap size the dispatchers use.
#define FFS_DECODER_BODIES
#include "ffs_device.cuh"

namespace fgpu {

#define FFS_PAIR_INST(MM)                                                                                            \
    template __device__ uint4 pair_round<MM, false>(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t,     \
                                                     uint32_t, uint32_t, uint32_t, int, uint32_t);                  \
    template __device__ uint4 pair_round<MM, true>(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t,      \
                                                    uint32_t, uint32_t, uint32_t, int, uint32_t);
FFS_PAIR_INST(1) FFS_PAIR_INST(2) FFS_PAIR_INST(3) FFS_PAIR_INST(4) FFS_PAIR_INST(5) FFS_PAIR_INST(6)
FFS_PAIR_INST(7) FFS_PAIR_INST(8) FFS_PAIR_INST(9) FFS_PAIR_INST(10) FFS_PAIR_INST(11) FFS_PAIR_INST(12)
FFS_PAIR_INST(13) FFS_PAIR_INST(14) FFS_PAIR_INST(15) FFS_PAIR_INST(16) FFS_PAIR_INST(kMaxM)
#undef FFS_PAIR_INST

}  // namespace fgpu
